"""The C-ABI library builds, loads without a GPU and exports every function include/relo.h
declares; the ctypes binding names exactly those functions.  No compute call is made."""
import ctypes
import os
import re

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            s = open(os.path.join(inc, f)).read()
            s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
            s = re.sub(r"//[^\n]*", "", s)
            names |= set(re.findall(r"\b(relo_[a-z0-9_]+)\s*\(", s))
    return names


def test_header_declares_the_binding_names():
    declared = _declared()
    assert len(declared) > 40
    assert declared == set(B.EXPORTED)


def test_library_loads_and_exports_every_declared_function():
    build.build()
    L = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert B.lib() is not None


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "relo.h"

static void* fake_alloc(size_t bytes, void* ctx) { (void)bytes; (void)ctx; return NULL; }
static void fake_free(void* ptr, void* ctx) { (void)ptr; (void)ctx; }

int main(void) {
  relo_pose_graph* g = NULL;
  if (relo_pose_graph_create(0, &g) != RELO_EINVAL) return 1;      /* bad size rejected */
  if (relo_pose_graph_create(3, &g) != RELO_OK || !g) return 2;
  double T[16] = {1, 0, 0, 0.5, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  int32_t size = 0;
  if (relo_pose_graph_add_sample(g, 0, 1, T, &size) != RELO_OK || size != 1) return 3;
  if (relo_pose_graph_add_sample(g, 1, 0, T, &size) != RELO_OK || size != 1) return 4;  /* inverse: other cluster */
  T[3] = 0.52;
  if (relo_pose_graph_add_sample(g, 0, 1, T, &size) != RELO_OK || size != 2) return 5;
  double poses[3 * 16];
  int32_t in_graph[3];
  double eps = -1;
  if (relo_pose_graph_optimise(g, poses, in_graph, &eps) != RELO_OK) return 6;
  if (!in_graph[0] || !in_graph[1] || in_graph[2]) return 7;
  if (poses[16 + 3] < 0.509 || poses[16 + 3] > 0.511) return 8;     /* the blend of 0.50 and 0.52 */
  if (relo_pose_graph_add_sample(g, 1, 1, T, NULL) != RELO_EINVAL) return 9;
  relo_pose_graph_destroy(g);
  relo_schedule s;
  memset(&s, 0, sizeof s);
  if (relo_batch_set_schedule(NULL, &s) != RELO_EINVAL || strlen(relo_last_error()) == 0) return 10;
  if (relo_set_allocator(NULL, NULL, NULL) != RELO_OK) return 11;          /* back to cudaMalloc */
  if (relo_set_allocator(fake_alloc, NULL, NULL) != RELO_EINVAL) return 12; /* both or neither */
  if (relo_set_allocator(NULL, fake_free, NULL) != RELO_EINVAL) return 13;
  if (relo_set_allocator(fake_alloc, fake_free, &s) != RELO_OK) return 14;
  if (relo_set_allocator(NULL, NULL, NULL) != RELO_OK) return 15;
  printf("ok\n");
  return 0;
}
"""


def test_a_c_program_uses_the_abi(tmp_path):
    """The header is plain C99 and the library links into a C program: host-only calls (the pose
    graph, argument errors, relo_last_error and relo_set_allocator) behave as documented without
    a GPU."""
    import subprocess
    build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(B.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lrelo", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == "ok"


def test_set_allocator_arguments():
    """Host side of relo_set_allocator: both callbacks or neither (no allocation is made here)."""
    import pytest
    with pytest.raises(ValueError):
        B.set_allocator(lambda n: 0)
    L = B.lib()
    assert L.relo_set_allocator(B.ALLOC_FN(lambda n, c: None), B.FREE_FN(), None) == B.EINVAL
    B.set_allocator(lambda n: 0, lambda p: None)
    B.set_allocator()


LAYOUTS = {"relo_intrinsics": B.Intrinsics, "relo_train_params": B.TrainParams,
           "relo_ransac_params": B.RansacParams, "relo_pose_result": B.PoseResult, "relo_attempt": B.Attempt,
           "relo_schedule": B.Schedule, "relo_server_params": B.ServerParams, "relo_server_stats": B.ServerStats}


def test_binding_structs_match_the_header_layouts(tmp_path):
    """Every struct the binding passes by pointer has the header's size and field offsets, as a C
    compiler lays them out (a C program prints sizeof / offsetof)."""
    import subprocess
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "relo.h"', "int main(void) {"]
    for cname, cls in LAYOUTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for cname, cls in LAYOUTS.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)

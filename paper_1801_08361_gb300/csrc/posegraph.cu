// posegraph.cu -- the host consumer of relative transform samples (Sec. 3.3.2): incremental
// clustering per pair of sub-scenes, dual-quaternion blending of each confident pair's largest
// cluster, the pose graph of agent 0's connected component, and Levenberg-Marquardt on the
// error of Sec. 3.3.2; plus the candidate score Phi of Sec. 3.3.1 that schedules attempts.
//
// Readings (the paper states the rules, not every detail): samples of (a, b) and (b, a) share
// one set of clusters for the unordered pair, stored in the canonical direction aT_b with a < b
// (a reversed sample is inverted); "within 20 degrees and 10 cm" compares the
// rotation angle of R1 R2^T and the distance of the translations; blending weights the cluster's
// samples equally, with each quaternion's sign aligned to the first sample's before summing
// (Kavan et al., dual quaternion linear blending); v(T) takes the quaternion with w >= 0; LM
// minimises the sum of squared residual components (epsilon, the sum of the residual norms, is
// reported as printed); agent 0's global pose is the identity (the gauge).  Host code only.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/relo.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Rigid {
  double R[9];
  double t[3];
};

Rigid from_mat(const double* m) {
  Rigid T;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T.R[3 * i + j] = m[4 * i + j];
    T.t[i] = m[4 * i + 3];
  }
  return T;
}

void to_mat(const Rigid& T, double* m) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) m[4 * i + j] = T.R[3 * i + j];
    m[4 * i + 3] = T.t[i];
  }
  m[12] = m[13] = m[14] = 0.0;
  m[15] = 1.0;
}

Rigid mul(const Rigid& A, const Rigid& B) {
  Rigid C;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A.R[3 * i + k] * B.R[3 * k + j];
      C.R[3 * i + j] = s;
    }
    double s = A.t[i];
    for (int k = 0; k < 3; ++k) s += A.R[3 * i + k] * B.t[k];
    C.t[i] = s;
  }
  return C;
}

Rigid inverse(const Rigid& A) {
  Rigid B;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B.R[3 * i + j] = A.R[3 * j + i];
  for (int i = 0; i < 3; ++i) B.t[i] = -(B.R[3 * i] * A.t[0] + B.R[3 * i + 1] * A.t[1] + B.R[3 * i + 2] * A.t[2]);
  return B;
}

Rigid identity() {
  Rigid T{};
  T.R[0] = T.R[4] = T.R[8] = 1.0;
  return T;
}

// Rotation angle (radians) of R1 R2^T.
double angle_between(const double* R1, const double* R2) {
  double tr = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) tr += R1[3 * i + k] * R2[3 * i + k];
  return std::acos(std::max(-1.0, std::min(1.0, (tr - 1.0) / 2.0)));
}

double dist3(const double* a, const double* b) {
  return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
}

// Unit quaternion (w, x, y, z) of a rotation matrix, w >= 0 (Shepperd's method: the largest of
// the four squared components decides which formula is stable).
void quat_from_R(const double* R, double* q) {
  const double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr > 0.0) {
    const double s = std::sqrt(tr + 1.0) * 2.0;
    w = 0.25 * s;
    x = (R[7] - R[5]) / s;
    y = (R[2] - R[6]) / s;
    z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const double s = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;
    w = (R[7] - R[5]) / s;
    x = 0.25 * s;
    y = (R[1] + R[3]) / s;
    z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const double s = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;
    w = (R[2] - R[6]) / s;
    x = (R[1] + R[3]) / s;
    y = 0.25 * s;
    z = (R[5] + R[7]) / s;
  } else {
    const double s = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;
    w = (R[3] - R[1]) / s;
    x = (R[2] + R[6]) / s;
    y = (R[5] + R[7]) / s;
    z = 0.25 * s;
  }
  const double n = std::sqrt(w * w + x * x + y * y + z * z), sg = w < 0.0 ? -1.0 : 1.0;
  q[0] = sg * w / n;
  q[1] = sg * x / n;
  q[2] = sg * y / n;
  q[3] = sg * z / n;
}

void R_from_quat(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

void qmul(const double* a, const double* b, double* c) {
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Dual quaternion linear blending with equal weights (Kavan et al. 2006): real parts q_i (signs
// aligned with the first), dual parts d_i = 1/2 (0, t_i) q_i; the sum is normalised by its real
// part's norm; the blended translation is 2 d q*.
Rigid blend(const std::vector<Rigid>& S) {
  double br[4] = {0, 0, 0, 0}, bd[4] = {0, 0, 0, 0}, q0[4];
  for (size_t i = 0; i < S.size(); ++i) {
    double q[4];
    quat_from_R(S[i].R, q);
    if (i == 0) std::copy(q, q + 4, q0);
    if (q[0] * q0[0] + q[1] * q0[1] + q[2] * q0[2] + q[3] * q0[3] < 0.0)
      for (double& v : q) v = -v;
    const double tq[4] = {0.0, S[i].t[0], S[i].t[1], S[i].t[2]};
    double d[4];
    qmul(tq, q, d);
    for (int k = 0; k < 4; ++k) {
      br[k] += q[k];
      bd[k] += 0.5 * d[k];
    }
  }
  const double n = std::sqrt(br[0] * br[0] + br[1] * br[1] + br[2] * br[2] + br[3] * br[3]);
  for (int k = 0; k < 4; ++k) {
    br[k] /= n;
    bd[k] /= n;
  }
  Rigid T;
  R_from_quat(br, T.R);
  const double conj[4] = {br[0], -br[1], -br[2], -br[3]};
  double tq[4];
  qmul(bd, conj, tq);
  for (int k = 0; k < 3; ++k) T.t[k] = 2.0 * tq[1 + k];
  return T;
}

// v(T): imaginary part of T's rotation quaternion (w >= 0), then T's translation.
void vee(const Rigid& T, double* v) {
  double q[4];
  quat_from_R(T.R, q);
  v[0] = q[1];
  v[1] = q[2];
  v[2] = q[3];
  v[3] = T.t[0];
  v[4] = T.t[1];
  v[5] = T.t[2];
}

// exp of the rotation vector w (Rodrigues), applied on the left: R <- exp([w]) R.
void rotate_left(double* R, const double* w) {
  const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double E[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (th > 0.0) {
    const double k[3] = {w[0] / th, w[1] / th, w[2] / th}, s = std::sin(th), c = 1.0 - std::cos(th);
    const double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double sum = 0.0;
        for (int m = 0; m < 3; ++m) sum += K[3 * i + m] * K[3 * m + j];
        K2[3 * i + j] = sum;
      }
    for (int i = 0; i < 9; ++i) E[i] += s * K[i] + c * K2[i];
  }
  double out[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double sum = 0.0;
      for (int m = 0; m < 3; ++m) sum += E[3 * i + m] * R[3 * m + j];
      out[3 * i + j] = sum;
    }
  std::copy(out, out + 9, R);
}

// Solves the symmetric positive definite system A x = b (n x n, row-major) by Cholesky.
bool cholesky_solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= A[(size_t)i * n + k] * b[k];
    b[i] = s / A[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= A[(size_t)k * n + i] * b[k];
    b[i] = s / A[(size_t)i * n + i];
  }
  return true;
}

struct Edge {
  int a, b;
  Rigid T;  // aT_b
};

}  // namespace

struct relo_pose_graph {
  int n = 0;
  // clusters[pair] : list of clusters, each a list of samples aT_b (a < b)
  std::vector<std::vector<std::vector<Rigid>>> clusters;
  std::vector<std::vector<double>> tried;  // per ordered (a, b): local frame poses tried (12 doubles each)
  std::vector<int> optimised;              // scenes with an optimised global pose (last optimisation)
  int pair_index(int a, int b) const { return a * n + b; }
};

namespace {

constexpr int kConfidentN = 2;            // Sec. 3.3.1: N = 2
constexpr double kClusterAngle = 20.0 * kPi / 180.0, kClusterDist = 0.10;  // Sec. 4.2.4
constexpr double kHomogAngle = 5.0 * kPi / 180.0, kHomogDist = 0.05;      // Sec. 3.3.1
constexpr double kHomogPenalty = 5.0;

size_t largest(const std::vector<std::vector<Rigid>>& cl) {
  size_t m = 0;
  for (const auto& c : cl) m = std::max(m, c.size());
  return m;
}

// LM on the squared residuals r_e = v(gT_b^-1 gT_a aT_b) over the edges; gT of nodes[0] fixed.
double optimise_graph(const std::vector<int>& nodes, const std::vector<Edge>& edges, std::vector<Rigid>& g,
                      int max_iter) {
  const int m = (int)nodes.size() - 1;  // free nodes
  std::vector<int> slot(g.size(), -1);
  for (int i = 1; i <= m; ++i) slot[nodes[i]] = i - 1;
  auto residuals = [&](const std::vector<Rigid>& G, std::vector<double>& r) {
    r.assign(edges.size() * 6, 0.0);
    for (size_t e = 0; e < edges.size(); ++e) {
      const Rigid D = mul(mul(inverse(G[edges[e].b]), G[edges[e].a]), edges[e].T);
      vee(D, &r[6 * e]);
    }
  };
  auto sq = [](const std::vector<double>& r) { return std::inner_product(r.begin(), r.end(), r.begin(), 0.0); };
  auto perturb = [&](std::vector<Rigid>& G, int node, const double* dx) {
    rotate_left(G[node].R, dx);
    for (int k = 0; k < 3; ++k) G[node].t[k] += dx[3 + k];
  };
  std::vector<double> r;
  residuals(g, r);
  double cost = sq(r), lambda = 1e-3;
  const int P = 6 * m;
  if (P == 0) return cost;
  for (int it = 0; it < max_iter; ++it) {
    // Jacobian by central differences (the graphs are small: one node per sub-scene)
    std::vector<double> J(r.size() * P, 0.0), rp, rm;
    const double h = 1e-6;
    for (int i = 1; i <= m; ++i)
      for (int k = 0; k < 6; ++k) {
        double dx[6] = {0, 0, 0, 0, 0, 0};
        std::vector<Rigid> Gp(g), Gm(g);
        dx[k] = h;
        perturb(Gp, nodes[i], dx);
        dx[k] = -h;
        perturb(Gm, nodes[i], dx);
        residuals(Gp, rp);
        residuals(Gm, rm);
        for (size_t q = 0; q < r.size(); ++q) J[q * P + 6 * (i - 1) + k] = (rp[q] - rm[q]) / (2 * h);
      }
    std::vector<double> JtJ((size_t)P * P, 0.0), Jtr(P, 0.0);
    for (size_t q = 0; q < r.size(); ++q)
      for (int i = 0; i < P; ++i) {
        const double ji = J[q * P + i];
        if (ji == 0.0) continue;
        Jtr[i] += ji * r[q];
        for (int j = 0; j < P; ++j) JtJ[(size_t)i * P + j] += ji * J[q * P + j];
      }
    bool improved = false;
    for (int tries = 0; tries < 10 && !improved; ++tries) {
      std::vector<double> A(JtJ), b(P);
      for (int i = 0; i < P; ++i) {
        A[(size_t)i * P + i] += lambda * std::max(JtJ[(size_t)i * P + i], 1e-12);
        b[i] = -Jtr[i];
      }
      if (!cholesky_solve(A, b, P)) {
        lambda *= 10.0;
        continue;
      }
      std::vector<Rigid> G2(g);
      for (int i = 1; i <= m; ++i) perturb(G2, nodes[i], &b[6 * (i - 1)]);
      std::vector<double> r2;
      residuals(G2, r2);
      const double c2 = sq(r2);
      if (c2 < cost) {
        const double drop = cost - c2;
        g.swap(G2);
        r.swap(r2);
        cost = c2;
        lambda = std::max(lambda * 0.1, 1e-12);
        improved = true;
        if (drop < 1e-16 * (1.0 + cost)) return cost;
      } else {
        lambda *= 10.0;
      }
    }
    if (!improved) break;
  }
  return cost;
}

}  // namespace

extern "C" {

relo_status relo_pose_graph_create(int32_t n_scenes, relo_pose_graph** out) {
  if (!out) return RELO_EINVAL;
  *out = nullptr;
  if (n_scenes < 1 || n_scenes > 4096) return RELO_EINVAL;
  relo_pose_graph* g = new relo_pose_graph();
  g->n = n_scenes;
  g->clusters.assign((size_t)n_scenes * n_scenes, {});
  g->tried.assign((size_t)n_scenes * n_scenes, {});
  g->optimised.assign(n_scenes, 0);
  *out = g;
  return RELO_OK;
}

void relo_pose_graph_destroy(relo_pose_graph* g) { delete g; }

relo_status relo_pose_graph_add_sample(relo_pose_graph* g, int32_t a, int32_t b, const double aTb[16],
                                       int32_t* cluster_size) {
  if (!g || !aTb || a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) return RELO_EINVAL;
  Rigid T = from_mat(aTb);
  if (a > b) {  // canonical direction: the smaller index first
    T = inverse(T);
    std::swap(a, b);
  }
  auto& cl = g->clusters[g->pair_index(a, b)];
  size_t at = cl.size();
  for (size_t c = 0; c < cl.size() && at == cl.size(); ++c)
    for (const Rigid& s : cl[c])
      if (angle_between(s.R, T.R) <= kClusterAngle && dist3(s.t, T.t) <= kClusterDist) {
        at = c;
        break;
      }
  if (at == cl.size()) cl.push_back({});
  cl[at].push_back(T);
  if (cluster_size) *cluster_size = (int32_t)cl[at].size();
  return RELO_OK;
}

relo_status relo_pose_graph_optimise(relo_pose_graph* g, double* global_poses, int32_t* in_graph,
                                     double* epsilon) {
  if (!g || !global_poses || !in_graph) return RELO_EINVAL;
  const int n = g->n;
  // G': confident pairs, each with the blend of its largest cluster
  std::vector<Edge> all;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      const auto& cl = g->clusters[g->pair_index(a, b)];
      if ((int)largest(cl) < kConfidentN) continue;
      size_t best = 0;
      for (size_t c = 1; c < cl.size(); ++c)
        if (cl[c].size() > cl[best].size()) best = c;  // the first of equal largest clusters
      all.push_back({a, b, blend(cl[best])});
    }
  // connected component of scene 0 (breadth first), global poses along the search tree
  std::vector<Rigid> G(n, identity());
  std::vector<int> seen(n, 0), nodes = {0};
  seen[0] = 1;
  for (size_t q = 0; q < nodes.size(); ++q) {
    const int u = nodes[q];
    for (const Edge& e : all) {
      if (e.a == u && !seen[e.b]) {  // gT_b = gT_a aT_b
        G[e.b] = mul(G[u], e.T);
        seen[e.b] = 1;
        nodes.push_back(e.b);
      } else if (e.b == u && !seen[e.a]) {  // gT_a = gT_b (aT_b)^-1
        G[e.a] = mul(G[u], inverse(e.T));
        seen[e.a] = 1;
        nodes.push_back(e.a);
      }
    }
  }
  std::vector<Edge> edges;
  for (const Edge& e : all)
    if (seen[e.a] && seen[e.b]) edges.push_back(e);
  optimise_graph(nodes, edges, G, 100);
  double eps = 0.0;
  for (const Edge& e : edges) {
    double v[6];
    vee(mul(mul(inverse(G[e.b]), G[e.a]), e.T), v);
    double s = 0.0;
    for (double x : v) s += x * x;
    eps += std::sqrt(s);
  }
  for (int s = 0; s < n; ++s) {
    in_graph[s] = seen[s];
    g->optimised[s] = seen[s];
    to_mat(seen[s] ? G[s] : identity(), global_poses + 16 * (size_t)s);
  }
  if (epsilon) *epsilon = eps;
  return RELO_OK;
}

relo_status relo_pose_graph_mark_tried(relo_pose_graph* g, int32_t a, int32_t b, const double pose_in_b[16]) {
  if (!g || !pose_in_b || a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) return RELO_EINVAL;
  const Rigid T = from_mat(pose_in_b);
  auto& v = g->tried[g->pair_index(a, b)];
  v.insert(v.end(), T.R, T.R + 9);
  v.insert(v.end(), T.t, T.t + 3);
  return RELO_OK;
}

relo_status relo_pose_graph_score(const relo_pose_graph* g, int32_t a, int32_t b, const double pose_in_b[16],
                                  double* score) {
  if (!g || !pose_in_b || !score || a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) return RELO_EINVAL;
  const double phi_new = (g->optimised[a] != g->optimised[b]) ? 1.0 : 0.0;
  const auto& cl = g->clusters[g->pair_index(std::min(a, b), std::max(a, b))];
  const double phi_conf = std::max(0.0, (double)largest(cl) - kConfidentN);
  const Rigid T = from_mat(pose_in_b);
  double phi_homog = 0.0;
  const auto& v = g->tried[g->pair_index(a, b)];
  for (size_t k = 0; k + 12 <= v.size(); k += 12)
    if (angle_between(&v[k], T.R) <= kHomogAngle && dist3(&v[k + 9], T.t) <= kHomogDist) {
      phi_homog = kHomogPenalty;
      break;
    }
  *score = phi_new - phi_conf - phi_homog;
  return RELO_OK;
}

relo_status relo_pose_graph_cluster_blend(const relo_pose_graph* g, int32_t a, int32_t b, int32_t c,
                                          double aTb[16]) {
  if (!g || !aTb || a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) return RELO_EINVAL;
  const auto& cl = g->clusters[g->pair_index(std::min(a, b), std::max(a, b))];
  if (c < 0 || c >= (int32_t)cl.size()) return RELO_EINVAL;
  const Rigid T = blend(cl[c]);
  to_mat(a < b ? T : inverse(T), aTb);
  return RELO_OK;
}

int32_t relo_pose_graph_cluster_count(const relo_pose_graph* g, int32_t a, int32_t b, int32_t* sizes,
                                      int32_t capacity) {
  if (!g || a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) return -1;
  const auto& cl = g->clusters[g->pair_index(std::min(a, b), std::max(a, b))];
  for (int32_t c = 0; c < (int32_t)cl.size() && c < capacity; ++c)
    if (sizes) sizes[c] = (int32_t)cl[c].size();
  return (int32_t)cl.size();
}

}  // extern "C"

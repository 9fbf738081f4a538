"""Named workload presets: the five configurations the framework is measured and tested on, with
the parameters each one fixes.  Every value is a plain number; the synthetic scenes they name come
from paper_1801_08361_gb300.synth.

- TINY: a 4 x 4 x 3 m room with 20 boxes, one 320 x 240 query, a depth-10 forest, 64 hypotheses.
- HOUSE: the paper-sized workload of the benchmark: a 10 x 8 x 3 m house of six rooms, 640 x 480
  queries with quadratic depth noise, a depth-15 forest, 1024 hypotheses (Sec. 4.3.2 sizes).
- FRAGMENTS: eight sub-scenes cut from the house, each in its own frame; all 56 ordered pairs per
  batch with mixed query sizes and hypothesis counts.
- LEARNED: the house with the cell regressor trained online (2000 steps of 16 views; learning
  rate 1e-3 after a linear warm-up over the first 5 % of the steps, cosine decay to zero).
- SERVING: single attempts from 4-16 agents at Poisson arrival rates, batched by the server.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    world: str                   # synth world: "room" (room_world(1)) or "house" (house_world(2))
    log2_buckets: int
    sizes: tuple                 # query (width, height) choices
    trees: int
    depth: int
    max_modes: int
    reservoir: int
    hypotheses: tuple            # K, or the range (lo, hi) it is drawn from
    batch_pixels: int            # B pixels added per preemptive round
    max_tries: int = 10000
    train_per_room: int = 16
    extra: dict = field(default_factory=dict)


TINY = Workload("tiny", "room", 16, ((320, 240),), 5, 10, 10, 64, (64,), 500, train_per_room=10)
HOUSE = Workload("house", "house", 20, ((640, 480),), 5, 15, 10, 1024, (1024,), 64)
FRAGMENTS = Workload("fragments", "house", 19, ((320, 240), (480, 360), (640, 480)), 5, 13, 10, 512, (256, 1024), 64,
                     extra={"fragments": 8, "pairs": 56})
LEARNED = Workload("learned", "house", 20, ((640, 480),), 5, 15, 10, 1024, (1024,), 64,
                   extra={"train_steps": 2000, "train_batch": 16, "lr": 1e-3, "warmup": 0.05,
                          "origin": (5.0, 4.0, 1.5)})
SERVING = Workload("serving", "house", 20, ((640, 480),), 5, 15, 10, 1024, (1024,), 64,
                   extra={"agents": (8, 16), "offered_per_s": (200.0, 4000.0), "max_batch": 64,
                          "max_wait_us": 2000, "slots": 512})

ALL = {w.name: w for w in (TINY, HOUSE, FRAGMENTS, LEARNED, SERVING)}


def learning_rate(step: int, steps: int, peak: float, warmup: float) -> float:
    """The online training's schedule: linear warm-up over the first ``warmup`` fraction of the
    steps, then a cosine decay from ``peak`` towards zero."""
    import math
    w = max(1.0, warmup * steps)
    return peak * min(1.0, (step + 1) / w) * 0.5 * (1.0 + math.cos(math.pi * step / steps))

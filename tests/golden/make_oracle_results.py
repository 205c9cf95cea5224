"""Write the FP64 oracle's full results for the full-size frames, so that the
GPU parity tests can compare modes and label maps element by element without
re-running the oracle (a minute per 512x512 frame, about 25 minutes for the
three-frame tracking stack on 8 cores). Calls only oracle/ and synth/.

    python tests/golden/make_oracle_results.py [c2] [c3]

Each <name>_oracle_result.npz holds, for synth.frame_c2(seed=0) or
synth.stack_c3(seed=0) with the default configuration (c = 0.9, tol 1e-6,
OSOP gamma 0.9, N_initial 128, L 2, H 8, P 0.99, merge_cos = c):
  modes      float64 [K, 16]  kept modes in keep order (Algorithm 2, prune/merge)
  support    int64 [K]        window size of each mode's converging update
  labels     int32 [H*W]      argmax label per pixel, -1 background (Algorithm 2, labelling)
  margin_gt  uint8 packbits   per pixel: top-1 minus top-2 cosine > 1e-5
  seed_log   int32 [seeds]    foreground index of every seed in draw order
  round_log  int64 [rounds,4] N requested, seeds drawn, modes kept, uncovered
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
FRAMES = {"c2": lambda: synth.frame_c2(seed=0), "c3": lambda: synth.stack_c3(seed=0)}
SAFE_MARGIN = 1e-5


def write(name):
    f = FRAMES[name]()
    t0 = time.time()
    r = oracle.run(f.emb, f.mask)
    dt = time.time() - t0
    margin = np.nan_to_num(r.label_margin, nan=-1.0)
    out = os.path.join(HERE, f"{name}_oracle_result.npz")
    np.savez_compressed(out, modes=r.modes, support=r.support, labels=r.labels.astype(np.int32),
                        margin_gt=np.packbits(margin > SAFE_MARGIN), n_pixels=np.int64(r.labels.size),
                        seed_log=r.seed_log.astype(np.int32), round_log=r.round_log,
                        safe_margin=np.float64(SAFE_MARGIN))
    print(f"{name}: {r.modes.shape[0]} modes, {r.stats['seeds']} seeds, {dt:.0f} s -> {out}", flush=True)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(FRAMES)):
        write(name)

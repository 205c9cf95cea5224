"""Write c3_oracle_stats.json: the FP64 oracle's counters for the tracking
stack (three 512x512 frames clustered jointly) of the synthetic generator with
seed 0 (calls only oracle/ and synth/).

    python tests/golden/make_c3_oracle_stats.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

if __name__ == "__main__":
    f = synth.stack_c3(seed=0)
    t0 = time.time()
    r = oracle.run(f.emb, f.mask)
    out = dict(r.stats)
    out.update(frame="synth.stack_c3(seed=0)", n_fg=int(f.mask.sum()), seconds=round(time.time() - t0, 1),
               threads=len(os.sched_getaffinity(0)))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle_stats.json")
    json.dump(out, open(path, "w"), indent=1, sort_keys=True)
    print(json.dumps(out))

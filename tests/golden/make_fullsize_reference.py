"""Write the FP64 oracle signals of the full-size workloads.

    python tests/golden/make_fullsize_reference.py [fse|epi|all] [--threads N]

Calls only the oracle (``oracle.simulate`` with the exact memoised-transition
and ADC-recurrence shortcuts, each pinned against the direct form) on the
seeded 27,525,120-isochromat phantom, and stores the complex signal together
with the SHA-256 digests of the phantom and sequence it came from.  The GPU
full-size parity test refuses to compare against a file whose digests differ
from the inputs it generated.
"""

import argparse
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from mrsim_inputs import configs, phantom_digest, sequence_digest  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def make(name: str, threads: int):
    ph = configs.full_phantom()
    seq = configs.fse_sequence() if name == "fse" else configs.epi_sequence()
    t0 = time.time()
    sig, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True, n_threads=threads,
                             want_M=False)
    wall = time.time() - t0
    path = os.path.join(OUT, f"{name}_27m_oracle.npz")
    np.savez_compressed(path, signal=sig, phantom_digest=phantom_digest(ph),
                        sequence_digest=sequence_digest(seq), K=ph.K,
                        wall_s=wall, threads=threads, host=platform.machine())
    print(f"{name}: K={ph.K} samples={sig.size} wall={wall:.1f}s -> {path}", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="?", default="all", choices=["fse", "epi", "all"])
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    for n in (["fse", "epi"] if a.which == "all" else [a.which]):
        make(n, a.threads)

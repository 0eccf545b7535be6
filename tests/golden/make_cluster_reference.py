"""Write the oracle's clustering of the full-size parameter-mapping phantom.

    python tests/golden/make_cluster_reference.py

Calls only the oracle (``oracle.cluster.cluster_phantom``, 256 clusters, the
default feature scale and T2-weighted refit model) on the seeded
27,525,120-isochromat phantom ``configs.mapped_27m()`` and stores what the GPU
full-size test compares: the SHA-256 of the cluster labels, the FP64 centres,
the split history, the cluster sizes and the refitted M0 at every 99,991st
isochromat, with the digest of the phantom they came from.
"""

import hashlib
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cluster as oc  # noqa: E402
from mrsim_inputs import configs, phantom_digest  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))
N_CLUSTERS = 256
STRIDE = 99991


def main():
    ph = configs.mapped_27m()
    t0 = time.time()
    r = oc.cluster_phantom(ph, N_CLUSTERS)
    wall = time.time() - t0
    labels = np.ascontiguousarray(r.labels, np.int32)
    np.savez_compressed(
        os.path.join(OUT, "cluster_mapped_27m_oracle.npz"),
        phantom_digest=phantom_digest(ph), n_clusters=N_CLUSTERS,
        labels_sha256=hashlib.sha256(labels.tobytes()).hexdigest(),
        centres=r.centres, history=np.asarray(r.history, np.int32),
        sizes=np.bincount(labels, minlength=len(r.centres)),
        m0_index=np.arange(0, ph.K, STRIDE), m0=r.phantom.M0[::STRIDE],
        wall_s=wall, host=platform.machine())
    print(f"{len(r.centres)} clusters in {wall:.1f} s")


if __name__ == "__main__":
    main()

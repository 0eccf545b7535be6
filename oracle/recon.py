"""Image reconstruction of Cartesian k-space (reference for the CUDA path).

TEST INFRASTRUCTURE ONLY: loaded by the tests, never by the library.

The simulated signal of a Cartesian sequence is, per Eq. 6, samples of the
Fourier transform of the transverse magnetization; the image is its centred,
normalised inverse DFT.  The paper reconstructs its SE and FSE data with an FFT
and its EPI data by gridding ("Simulations #1"); the EPI here samples only on
the gradient flat-tops, so after reversing every other line its samples lie on
the Cartesian grid and gridding reduces to the same DFT.  Each acquisition
line is put into its k-space row and columns
(``mrsim_inputs.kspace_layout``), then

    image[y, x] = 1/(N M) sum_{ky, kx} K[ky, kx] exp(+i 2 pi ((kx - N/2)(x - N/2) / N
                                                         + (ky - M/2)(y - M/2) / M))

for even N (readout) and M (lines), i.e. fftshift(ifft2(ifftshift(K))).  The
library FFT is the only step used.
"""

import numpy as np


def kspace(signal, layout):
    n_ro, n_pe = layout["n_ro"], layout["n_pe"]
    S = np.asarray(signal, np.complex128).reshape(-1, n_ro)
    K = np.zeros((n_pe, n_ro), np.complex128)
    i = np.arange(n_ro)
    for a in range(S.shape[0]):
        cols = (int(layout["col0"][a]) + int(layout["dir"][a]) * i) % n_ro
        K[int(layout["row"][a]), cols] += S[a]
    return K


def recon_cartesian(signal, layout):
    """Complex image [n_pe, n_ro] of one coil's signal [n_lines * n_ro]."""
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(kspace(signal, layout))))

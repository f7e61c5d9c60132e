"""Exact projections with a plain definition -- TEST INFRASTRUCTURE ONLY.

project_2d_div_energy: family "C" (2-D velocity, discrete divergence with central
differences + kinetic energy, one frame at a time).  The feasible set of one frame is
{w : D w = 0} intersected with the sphere 1/2 dx^2 ||w||^2 = K, so the projection of eq. (2)
is the orthogonal projection P w_hat onto null(D) (a Leray projection) rescaled onto the
sphere:

    w* = R P w_hat / ||P w_hat||,   R = sqrt(2 K) / dx.

The KKT conditions of Appendix B, with L = 1/2||w - w_hat||^2 + lam_div^T D w
+ lam_K (1/2 dx^2 ||w||^2 - K), give
    (1 + lam_K dx^2) w* = P w_hat                 ->  lam_K = (||P w_hat|| / R - 1) / dx^2
    D^T lam_div = (I - P) w_hat                    ->  lam_div = (D D^T)^+ D w_hat + z,
with z in null(D^T) fixed so that lam_div = 0 on the four rows left out of the solve (cells
(0,0), (1,0), (0,1), (1,1), one per parity class; null(D^T) is spanned by the four parity
class indicators).

The periodic operators are diagonal in the discrete Fourier basis, with the central
difference symbol  d_x(p) = i sin(2 pi p / N) / dx  (library FFT as the only primitive).
Valid while P w_hat != 0 (otherwise every point of the sphere in null(D) is optimal).
"""
import numpy as np


def _symbols(N):
    dx = 1.0 / N
    s = np.sin(2.0 * np.pi * np.arange(N) / N) / dx
    sx = s[None, :]          # varies with i (x, axis 1)
    sy = s[:, None]          # varies with j (y, axis 0)
    return dx, sx, sy


def project_2d_frame(w_hat, K):
    """w_hat [2, N, N] (u, v with [j, i] = (y, x)); K = target kinetic energy.
    Returns (w [2, N, N], lam_div [N, N], lam_K)."""
    N = w_hat.shape[-1]
    dx, sx, sy = _symbols(N)
    U = np.fft.fft2(w_hat[0])
    V = np.fft.fft2(w_hat[1])
    s2 = sx * sx + sy * sy
    nz = s2 > 1e-12 * np.max(s2)
    # (D w)^ = i (sx U + sy V);  (D D^T)^ = s2;  D^T y ^ = conj(i s) y^ = -i s y^
    sdot = sx * U + sy * V
    ratio = np.where(nz, sdot / np.where(nz, s2, 1.0), 0.0)
    PU = U - sx * ratio
    PV = V - sy * ratio
    pu = np.real(np.fft.ifft2(PU))
    pv = np.real(np.fft.ifft2(PV))
    nrm = np.sqrt(np.sum(pu * pu) + np.sum(pv * pv))
    R = np.sqrt(2.0 * K) / dx
    w = np.stack([pu, pv]) * (R / nrm)
    lam_K = (nrm / R - 1.0) / (dx * dx)
    # lam_div = (D D^T)^+ D w_hat: (i sdot) / s2
    lam = np.real(np.fft.ifft2(1j * ratio))
    for (i, j) in ((0, 0), (1, 0), (0, 1), (1, 1)):
        lam[j % 2::2, i % 2::2] -= lam[j, i]
    return w, lam, lam_K


def project_2d(w_hat, params):
    """Batch: w_hat [B, nt, 2, N, N], params [B, 2] = (K0, r2).
    Returns (w, lam [B, nt*N*N + nt] in the family's nominal row order)."""
    w_hat = np.asarray(w_hat, np.float64)
    B, nt, _, N, _ = w_hat.shape
    t = np.arange(nt) / (nt - 1)
    w = np.empty_like(w_hat)
    lam = np.zeros((B, nt * N * N + nt))
    for b in range(B):
        for f in range(nt):
            K = params[b, 0] * np.exp(-params[b, 1] * t[f])
            wf, lf, lk = project_2d_frame(w_hat[b, f], K)
            w[b, f] = wf
            lam[b, f * N * N:(f + 1) * N * N] = lf.ravel()
            lam[b, nt * N * N + f] = lk
    return w, lam

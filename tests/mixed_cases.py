"""Inputs and references for the single-task checks of the mixed-precision
(TILEQR_TF32) updates, shared by the CPU test that pins the error bound and
the GPU test that applies it.

A DLARFB case: the reflectors V and T strip of a DGEQRT of one 128 x 128
tile, applied to a tile C.  A DSSRFB case: the reflectors of the DTSQRT of
a second tile into that R (Algorithm 2 on a 256 x 128 matrix), applied to
the pair [B'; C], B' being B after the DLARFB of the same step.  References
come from the CPU oracle (Algorithm 2's FP64 tile kernels, Sec. 3.2.1).

The bound: a 3xTF32 product (x = hi + lo, hi*hi + hi*lo + lo*hi, FP32
accumulation) carries about 2^-21 relative error per term; through the three
products of an update the output of column c then carries an error of a
small multiple of 2^-21 ||[B; C](:, c)||.  BOUND = 32 * 2^-21 per column.
"""
import numpy as np

import oracle
from paper_0709_1272_gb300 import inputs

BOUND = 32 * 2.0 ** -21


def larfb_case(ib, scale_exp=0, seed=31):
    A0 = inputs.normal_matrix(128, 128, seed=seed)
    C = np.ldexp(inputs.normal_matrix(128, 128, seed=seed + 3), scale_exp)
    f0 = oracle.tiled_qr(A0, 128, ib)
    V = np.array(f0.A, order="F")               # unit lower reflectors below R
    T = np.array(f0.T[:ib, :], order="F")
    ref = oracle.apply_qt(f0, C)
    return V, T, C, ref


def ssrfb_case(ib, scale_exp=0, seed=41):
    A0 = inputs.normal_matrix(128, 128, seed=seed)
    A1 = inputs.normal_matrix(128, 128, seed=seed + 1)
    B = np.ldexp(inputs.normal_matrix(128, 128, seed=seed + 2), scale_exp)
    C = np.ldexp(inputs.normal_matrix(128, 128, seed=seed + 3), scale_exp)
    f0 = oracle.tiled_qr(A0, 128, ib)
    f = oracle.tiled_qr(np.vstack([A0, A1]), 128, ib)
    V = np.array(f.A[128:, :], order="F")       # full DTSQRT reflector tile
    T = np.array(f.T[ib:2 * ib, :], order="F")
    Bp = oracle.apply_qt(f0, B)                 # the step's DLARFB of the top tile
    ref = oracle.apply_qt(f, np.vstack([B, C]))  # DLARFB then DSSRFB
    return V, T, Bp, C, ref


def column_error(out, ref, x):
    """max over columns of ||out(:,c) - ref(:,c)|| / ||x(:,c)||"""
    return float(np.max(np.linalg.norm(out - ref, axis=0) / np.linalg.norm(x, axis=0)))


# ---------------------------------------------------------------------------
# CPU emulation of the update's arithmetic (used only to show that BOUND
# separates 3xTF32 from products that drop a term).

def _tf32(x):
    x = np.asarray(x, dtype=np.float32)
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _product(a, b, terms):
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    ah, bh = _tf32(a), _tf32(b)
    al, bl = _tf32(a - ah), _tf32(b - bh)
    out = ah @ bh
    if "hl" in terms:
        out = out + ah @ bl
    if "lh" in terms:
        out = out + al @ bh
    return out.astype(np.float32)


def _full_t(Vfull, Tstrip, ib):
    """The b x b T of the reflectors, built column by column by the
    compact-WY rule T(0:j, j) = -tau_j T(0:j, 0:j) V(:, 0:j)^T v_j."""
    b = Vfull.shape[1]
    T = np.zeros((b, b))
    for j in range(b):
        tau = Tstrip[j % ib, j]
        T[j, j] = tau
        if j:
            T[:j, j] = -tau * T[:j, :j] @ (Vfull[:, :j].T @ Vfull[:, j])
    return T


def emulate_larfb(V, T, C, ib, terms=("hl", "lh")):
    Vu = np.tril(V, -1) + np.eye(128)
    Tf = _full_t(Vu, T, ib)
    P = _product(Vu.T, C, terms)
    W = _product(Tf.T, P, terms)
    D = _product(Vu, W, terms)
    return C - D.astype(np.float64)


def emulate_ssrfb(V, T, B, C, ib, terms=("hl", "lh")):
    Tf = _full_t(np.vstack([np.eye(128), V]), T, ib)
    P = _product(V.T, C, terms)
    Y = B.astype(np.float32) + P
    W = _product(Tf.T, Y, terms)
    D = _product(V, W, terms)
    return np.vstack([B - W.astype(np.float64), C - D.astype(np.float64)])

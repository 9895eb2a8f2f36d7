"""The error claim of the precision form's tensor-core integrals, checked on
the CPU by emulating their arithmetic in NumPy (no GPU, no library code):
operands rounded to float32, each split x = hi + lo with both parts exact in
TF32 (10 explicit significand bits, rounded to nearest on the magnitude), the
three products lo*hi + hi*lo + hi*hi per 32-point tile summed in float32, the
tile sums added in float64.  On the integrals of a small hanging-node mesh
(the oracle's orbitals and a set of smooth seeded fields) the emulated sums
stay within 1e-6 of the largest FP64 integral, and a single TF32 product
(no split) would not -- which is why the split is there."""
import numpy as np

from oracle import fem, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs

CASE = (-8.0, 8.0, 3, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
KT = 32


def tf32(x):
    """Round float32 values to TF32 (10 explicit bits) on the magnitude, as the
    library's tf32_round does: add half an ulp of TF32 to the bit pattern and
    clear the 13 low bits."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = tf32(x)
    lo = tf32((x - hi).astype(np.float32))
    return hi, lo


def emulated_contraction(A, B, three_products=True):
    """sum_f A[f, i] B[f, j] with the tensor-core recipe: float32 operands,
    32-row tiles, float32 tile sums (products of TF32 values are exact in
    float64, so the tile sum is formed in float64 and rounded once per
    product addition to float32), float64 across tiles."""
    F = A.shape[0]
    out = np.zeros((A.shape[1], B.shape[1]))
    for t0 in range(0, F, KT):
        a = A[t0:t0 + KT].astype(np.float32)
        b = B[t0:t0 + KT].astype(np.float32)
        ah, al = split(a)
        bh, bl = split(b)
        acc = np.zeros((A.shape[1], B.shape[1]), dtype=np.float32)
        pairs = ((al, bh), (ah, bl), (ah, bh)) if three_products else ((tf32(a), tf32(b)),)
        for k in range(a.shape[0]):
            for x, y in pairs:
                acc = (acc.astype(np.float64) + np.outer(x[k].astype(np.float64), y[k].astype(np.float64))
                       ).astype(np.float32)
        out += acc.astype(np.float64)
    return out


def test_split_products_are_exact_in_tf32():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1000).astype(np.float32) * 10.0 ** rng.uniform(-6, 6, 1000).astype(np.float32)
    hi, lo = split(x)
    for part in (hi, lo):
        assert np.all((part.view(np.uint32) & np.uint32(0x1FFF)) == 0)      # 13 low bits clear
    rel = np.abs(x.astype(np.float64) - hi - lo) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -21


def test_emulated_integrals_within_1e6_of_fp64():
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    n = 3
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], n), op.ML)
    rng = np.random.default_rng(17)
    r = np.sqrt(np.sum(om.Xm ** 2, axis=1))
    cols = np.stack([rng.uniform(0.2, 1.0) / np.sqrt(1.0 + r ** 2) for _ in range(n * n)], axis=1)
    # support points: masters then hanging points, values through the constraints
    pf = op.C @ (phi * (~om.boundary)[:, None])
    wf = op.C @ cols
    mf = op.m_f
    nn = n * n
    A = np.empty((len(mf), 2 * nn))
    for p in range(n):
        for q in range(n):
            d = mf * np.conj(pf[:, p]) * pf[:, q]
            A[:, 2 * (p * n + q)] = d.real
            A[:, 2 * (p * n + q) + 1] = d.imag
    ref = A.T @ wf                                     # FP64 contraction
    got = emulated_contraction(A, wf)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-6 * scale
    plain = emulated_contraction(A, wf, three_products=False)
    assert np.abs(plain - ref).max() > 1e-5 * scale   # one TF32 product is not enough

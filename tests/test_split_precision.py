"""Precision budget of the split forms, on the CPU: the operands of the three
contractions of Eq. 3 are split into 16-bit slices (bf16, or binary16 after a
power-of-two scaling), the kept slice products are summed exactly (FP64), and
chi is compared with the dense FP64 oracle.  This isolates the representation
error of each form from the tensor cores' accumulation (which rounds each MMA
step toward zero and is bounded by draining, not by the split):
  BF16x6 (3 bf16 slices, 6 products): ~1e-8
  FP16x3 (2 binary16 slices, 3 products): ~1e-7
  BF16x3 (2 bf16 slices, 3 products): ~5e-6, outside the 1e-6 bar
No code is shared with the CUDA path."""

import numpy as np
import pytest

from oracle import chi as oc
from synth import make_case


def _bf16(x):
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _split(x, kind, n):
    if kind == "fp16":
        m = np.abs(x).max()
        c = 2.0 ** (14 - np.ceil(np.log2(m))) if m > 0 else 1.0
        r = x * c
        out = []
        for _ in range(n):
            h = r.astype(np.float16).astype(np.float64)
            out.append(h / c)
            r = r - h
        return out
    r = x.copy()
    out = []
    for _ in range(n):
        h = _bf16(r)
        out.append(h)
        r = r - h
    return out


def _prod(a, b, f):
    # slice pairs (i, j) with i + j < number of slices
    n = len(a)
    return sum(f(a[i], b[j]) for i in range(n) for j in range(n) if i + j < n)


def _chi_split(t, go, gv, kind, n):
    nao = t.shape[0]
    ts, gos, gvs = _split(t, kind, n), _split(go, kind, n), _split(gv, kind, n)
    m = _prod(gos, ts, lambda g, x: np.einsum("ml,lsp->msp", g, x, optimize=True))
    nn = _prod(ts, gvs, lambda x, g: np.einsum("mnq,ns->msq", x, g, optimize=True))
    return -_prod(_split(m, kind, n), _split(nn, kind, n),
                  lambda a, b: a.reshape(nao * nao, -1).T @ b.reshape(nao * nao, -1))


@pytest.mark.parametrize("kind,n,lo,hi", [("bf16", 3, 0.0, 5e-8), ("fp16", 2, 1e-8, 3e-7),
                                          ("bf16", 2, 1e-6, 2e-5)])
def test_split_representation_error(kind, n, lo, hi):
    case = make_case("benzene", n_tau=3)
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data, 0.0)
    for j in range(len(case.tau)):
        go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[j])
        ref = oc.chi_dense_from_g(t, go, gv, oc.offsets(s.n_ao), oc.offsets(s.n_ri), 0.0, mirror=False)
        got = _chi_split(t, go, gv, kind, n)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert lo <= rel <= hi, f"{kind} x{n} tau {case.tau[j]}: {rel:.2e}"


def test_fp16_scaling_makes_the_error_magnitude_independent():
    """Scaling the tensor by 1e-7 or 1e7 (outside the binary16 range
    unscaled) leaves the FP16x3 relative error essentially unchanged (the
    power-of-two scales are exact; 1e+-7 changes the mantissas, hence the
    rounding pattern, a little)."""
    case = make_case("benzene", n_tau=2)
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data, 0.0)
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[1])
    errs = []
    for f in (1e-7, 1.0, 1e7):
        ref = oc.chi_dense_from_g(t * f, go, gv, oc.offsets(s.n_ao), oc.offsets(s.n_ri), 0.0,
                                  mirror=False)
        got = _chi_split(t * f, go, gv, "fp16", 2)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert max(errs) < 3e-7
    assert max(errs) / min(errs) < 1.1

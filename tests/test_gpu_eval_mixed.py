"""Interpolation with the mesh in mixed precision: the contraction of Eq.
u_tensor (Sec. 3.3) in double-float arithmetic on the FP32 pipe, against the
FP64 interpolation and the oracle.  Every value must lie within the
interpolation tolerance (1e-12 of the point's nodal scale) of the oracle's,
and within 1e-13 of that scale of the FP64 kernel's, the error bound of the
double-float contraction.  The nodal values are random (no smoothness, so
the Lebesgue constant's growth over the three stages is met in full), the
components are scaled by 1, 1e200 and 1e-200 (the per-component power-of-two
scaling keeps every value in the FP32 range) plus one all-zero component, and
the element types are
quads, hexes (order 7 on strongly deformed elements too), surface quads and
line elements (which keep the FP64 contraction), plus a field of another
order."""
import numpy as np
import pytest

import oracle
from paper_2501_12349_b300 import workloads as W
from parity_util import compare_eval, to_np

pytestmark = pytest.mark.gpu

CASES = {
    "quad2d_p3": lambda: (W.config1().coords, 2, 2, 3),
    "hex3d_p4": lambda: (W.hex_mesh(6, 4, 0.3), 3, 3, 4),
    "hex3d_p7_strong": lambda: (W.hex_mesh(3, 7, 0.6), 3, 3, 7),
    "sphere_p5": lambda: (W.cubed_sphere(3, 5), 3, 2, 5),
    "star_lines_p3": lambda: (W.star_lines(64, 3), 2, 1, 3),
}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def fp():
    import paper_2501_12349_b300 as f
    f.lib()
    return f


def _field(rng, NE, Nf, dr):
    f = rng.uniform(-1.0, 1.0, (4, NE, Nf ** dr))
    f[1] *= 1e200
    f[2] *= 1e-200
    f[3] = 0.0  # no exponent at all: scaled by 1, interpolates to 0
    return np.ascontiguousarray(f)


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_eval_matches_fp64_and_oracle(fp, torch, case):
    coords, d, dr, order = CASES[case]()
    N = order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(11)
    n = 20000
    elem = rng.integers(0, om.NE, n).astype(np.int32)
    rr = rng.uniform(-1.0, 1.0, (n, dr))
    rr[:50] = np.sign(rr[:50])            # on element boundaries and corners
    rr[50:100, 0] = oracle.gll_nodes(N)[1]  # on an interior node line
    # the find output of a forward-mapped point set, with some points not found
    code = np.zeros(n, np.int32)
    code[::97] = 2
    elem_in = np.where(code == 2, -1, elem).astype(np.int32)
    r_in = np.where(code[:, None] == 2, 0.0, rr)
    m = fp.Mesh(torch.from_numpy(np.ascontiguousarray(coords)).cuda(), d, dr, order)
    tc, te, tr = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (code, elem_in, r_in))
    for Nf in (N, max(2, N - 2)):
        field = _field(rng, om.NE, Nf, dr)
        tf = torch.from_numpy(field).cuda()
        order_f = None if Nf == N else Nf - 1
        m.set_precision(fp.FP_F64)
        u64 = to_np(m.eval(tc, te, tr, tf, order=order_f))
        m.set_precision(fp.FP_MIXED)
        udf = to_np(m.eval(tc, te, tr, tf, order=order_f))
        ne = Nf ** dr
        uo = om.eval(field, code, elem_in, r_in, field_N=None if Nf == N else Nf)
        compare_eval(field, om.NE, ne, elem_in, uo, udf, f"{case} Nf={Nf} mixed eval vs oracle")
        e = np.where(elem_in >= 0, elem_in, 0)
        nodal = np.abs(field).max(axis=2)[:, e]
        assert np.all(udf[3] == 0.0)
        nodal[3] = 1.0
        err = np.abs(udf - u64) / np.maximum(nodal, np.abs(u64))
        assert np.all(udf[:, code == 2] == 0.0)
        assert err.max() <= 1e-13, (case, Nf, float(err.max()))
        # the double-float path runs for quads, hexes and surfaces (its
        # rounding differs from FP64's somewhere); line elements, where it
        # would not pay, keep the FP64 contraction
        if dr >= 2:
            assert err.max() > 0.0, case
        else:
            assert np.array_equal(udf, u64), case
    assert m.device_status() == 0
    m.close()

"""The paper's size arithmetic and traffic/flop model (Sec. 3, Sec. 3.3) against the
values it prints (tests/golden/paper_model.txt)."""

import os

from paper_1607_04245_gb300 import perfmodel as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_model.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("="))
            vals[k] = int(v)
    return vals


def test_fig1_sizes():
    g = _golden()
    s = pm.TransposeSizes(N_b=g["fig1.N_b"], N_q=g["fig1.N_q"])
    assert s.N_t == g["fig1.N_t"]


def test_fig3_sizes():
    g = _golden()
    s = pm.TransposeSizes(N_b=g["fig3.N_b"], N_q=g["fig3.N_q"], N_comp=g["fig3.N_comp"], N_bl=g["fig3.N_bl"])
    assert s.N_bc == g["fig3.N_bc"]
    assert s.N_t == g["fig3.N_t"]
    assert s.N_tq == g["fig3.N_tq"]
    assert s.N_bt == g["fig3.N_bt"]
    # Fig. 1 caption: thread t0 handles 2 cells in the quadrature phase, 3 in the basis phase
    assert (s.N_sqc, s.N_sbc) == (2, 3)


def test_beta_poisson():
    g = _golden()
    for n_bl in (1, 2, 16, 32):
        s = pm.TransposeSizes(N_b=g["beta.N_b"], N_q=g["beta.N_q"], N_comp=g["beta.N_comp"], N_bl=n_bl)
        assert pm.beta(g["beta.d"], s) == (g["beta.num"], g["beta.den"])


def test_flops_per_cell_p1():
    # the model's per-cell flops for the two Laplacian workloads and the elasticity ones
    assert pm.flops_per_cell(2, 3, 1) == 246
    assert pm.flops_per_cell(3, 4, 1) == 824
    assert pm.flops_per_cell(2, 3, 2) == 492
    assert pm.flops_per_cell(3, 4, 3) == 2472


def test_collapsed_laplacian_flop_count():
    """The collapsed P1 Laplacian's count (87 flops per tetrahedron with 4 points, 30 per
    triangle with 3) against the paper model's per-point loops (824 per tetrahedron)."""
    from paper_1607_04245_gb300 import perfmodel

    assert perfmodel.collapsed_laplacian_flops(3, 4) == 87
    assert perfmodel.collapsed_laplacian_flops(2, 3) == 30
    assert perfmodel.flops_per_cell(3, 4, 1) > 9 * perfmodel.collapsed_laplacian_flops(3, 4)

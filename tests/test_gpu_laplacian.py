"""Parity of the CUDA Laplacian residual (fem_integrate_laplacian) with the CPU oracle.

Full-size workloads are compared element by element (the oracle finishes them in
about a second), plus ragged sizes, the scalar-load path, inverted cells, the
mixed form's float64 fallback and the degenerate cases.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, as_input, device_arrays, misaligned, rel_err, residual, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lap2d():
    return workloads.laplacian_square_case()  # 64x64 -> 8192 triangles


@pytest.fixture(scope="module")
def lap3d():
    return workloads.laplacian_cube_case()  # 1,572,864 tets


@pytest.mark.parametrize("prec", PRECS)
def test_square_8192_full(lap2d, prec):
    c, d = device_arrays(lap2d, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    err = rel_err(r, oracle.residual_for(c))
    print(f"lap2d 8192 {prec}: rel max-norm err {err:.3e}")
    assert err <= TOL[prec]
    if prec == "mixed":
        # against the float64 data the workload defines: the float32 storage of u and K
        # included, still inside the mixed form's tolerance
        err64 = rel_err(r, oracle.residual_for(lap2d))
        print(f"lap2d 8192 mixed vs the float64 inputs: {err64:.3e}")
        assert err64 <= TOL["mixed"]


@pytest.mark.parametrize("prec", PRECS)
def test_cube_1572864_full(lap3d, prec):
    c, d = device_arrays(lap3d, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    err = rel_err(r, oracle.residual_for(c))
    print(f"lap3d 1572864 {prec}: rel max-norm err {err:.3e}")
    assert err <= TOL[prec]
    if prec == "mixed":
        err64 = rel_err(r, oracle.residual_for(lap3d))  # the unrounded float64 u and K
        print(f"lap3d 1572864 mixed vs the float64 inputs: {err64:.3e}")
        assert err64 <= TOL["mixed"]
    # every element sum vanishes (r_0 is written as -(r_1 + ... + r_d))
    s = r.double().sum(0).abs().max().item()
    assert s <= (1e-15 if prec == "fp64" else 1e-6) * r.double().abs().max().item()


@pytest.mark.parametrize("n_cells", [1 << 16, 1 << 23])
def test_cube_sweep_ends_mixed(n_cells):
    case = workloads.laplacian_cube_case(n_cells)
    c, d = device_arrays(case, "mixed")
    r = residual(c, d, "mixed")
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL["mixed"]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_cells", [1, 2, 3, 5, 7, 4097, 6 * 7 ** 3 - 3])
@pytest.mark.parametrize("prec", PRECS)
def test_ragged_sizes(dim, n_cells, prec):
    base = workloads.laplacian_square_case(48) if dim == 2 else workloads.laplacian_cube_case(6 * 9 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_misaligned_pointers_take_scalar_path(lap2d, prec):
    c, d = device_arrays(lap2d, prec)
    ref = residual(c, d, prec).clone()
    d2 = dict(d, K=misaligned(d["K"]), conn=misaligned(d["conn"]))
    out = misaligned(torch.empty_like(ref))
    r = residual(c, d2, prec, out=out)
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]
    assert rel_err(r, ref.double().cpu().numpy()) <= TOL[prec]


def test_empty_mesh_is_noop(lap2d):
    c, d = device_arrays(lap2d, "fp64")
    conn = torch.empty((3, 0), dtype=torch.int32, device="cuda")
    K = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    r = fem.fem_integrate_laplacian(d["coords"], conn, d["u"], K, c.rule.points, c.rule.weights, prec="fp64")
    assert r.shape == (3, 0)


def _random_simplices(dim, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, dim + 1, dim))
    coords = X.reshape(-1, dim).T.copy()
    conn = np.arange(n * (dim + 1), dtype=np.int32).reshape(n, dim + 1).T.copy()
    return workloads.Mesh(dim, coords, conn)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inverted_cells_use_abs_det(dim, prec):
    """Random simplices, about half negatively oriented, some badly shaped."""
    mesh = _random_simplices(dim, 1000, seed=7)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(1)
    case = workloads.Case("laplacian", mesh, rule, rng.uniform(-1, 1, mesh.n_verts),
                          K=rng.lognormal(0, 1, (rule.n_q, mesh.n_cells)))
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_fallback_on_slivers(dim):
    """Nearly flat cells fail the shape test and take the float64 path."""
    base = workloads.laplacian_square_case(16) if dim == 2 else workloads.laplacian_cube_case(6 * 5 ** 3)
    mesh = base.mesh
    coords = mesh.coords.copy()
    # flatten every 7th cell: move its last vertex onto the plane/line of the others (almost)
    conn = mesh.conn.copy()
    V0 = coords.shape[1]
    sl = np.arange(0, mesh.n_cells, 7)
    new = []
    for c in sl:
        x = coords[:, conn[:, c]]
        p = x[:, :dim].mean(axis=1) + 1e-4 * (x[:, dim] - x[:, :dim].mean(axis=1))
        new.append(p)
        conn[dim, c] = V0 + len(new) - 1
    coords = np.concatenate([coords, np.stack(new, axis=1)], axis=1)
    u = np.concatenate([base.u, np.random.default_rng(2).uniform(-1, 1, len(new))])
    case = workloads.Case("laplacian", workloads.Mesh(dim, coords, conn), base.rule, u, K=base.K)
    c, d = device_arrays(case, "mixed")
    counts = fem.fem_check_mesh(d["coords"], d["conn"]).cpu().numpy()
    assert counts[0] == 0 and counts[1] == 0
    assert counts[2] >= len(sl)  # the slivers are flagged
    ref = oracle.residual_for(c)
    r = residual(c, d, "mixed")
    torch.cuda.synchronize()
    err = rel_err(r, ref)
    assert err <= TOL["mixed"], err
    old = fem.fem_get_mixed_threshold()
    try:
        fem.fem_set_mixed_threshold(2.0)  # every cell takes the float64 path
        r_all = residual(c, d, "mixed")
        torch.cuda.synchronize()
        assert rel_err(r_all, ref) <= 1e-6
    finally:
        fem.fem_set_mixed_threshold(old)


@pytest.mark.parametrize("scale,prec", [(1e-60, "fp64"), (1e-30, "fp64"), (1e30, "fp64"), (1e60, "fp64"),
                                        (1e-30, "mixed"), (1e30, "mixed")])
def test_extreme_coordinate_scales(scale, prec):
    """Coordinates scaled by up to 1e+-60: the float64 division by abs(det J) (a Newton-Raphson
    reciprocal with the exponent taken apart and put back) sees exponents near +-600, and the
    residual scales as scale^(d-2). In the mixed form det J leaves float32's range and every
    cell is recomputed in float64; its float32 outputs bound the scales it can take (the
    residual itself must be a normal float32). The collapsed P1 form multiplies
    Kbar / abs(det J) by n_j . h, which scales as scale^4 in 3D, so float64 coordinates must
    stay well inside 1e+-75."""
    base = workloads.laplacian_cube_case(6 * 8 ** 3)
    mesh = workloads.Mesh(3, base.mesh.coords * scale, base.mesh.conn)
    case = workloads.Case("laplacian", mesh, base.rule, base.u, K=base.K)
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    ref = oracle.residual_for(c)
    assert np.isfinite(ref).all() and np.abs(ref).max() > 0
    assert rel_err(r, ref) <= TOL[prec]


def test_constant_field_null_space(lap3d):
    for prec in ("fp64", "mixed"):
        c, d = device_arrays(lap3d, prec)
        d["u"].fill_(0.375)
        r = residual(c, d, prec)
        torch.cuda.synchronize()
        scale = np.abs(oracle.residual_for(as_input(lap3d, prec))).max()
        assert r.double().abs().max().item() <= (1e-15 if prec == "fp64" else 1e-7) * scale


def test_check_mesh_counts():
    case = workloads.laplacian_square_case(8)
    conn = case.mesh.conn.copy()
    conn[2, 5] = conn[1, 5]  # degenerate cell (repeated vertex)
    conn[0, 9] = case.n_verts + 3  # out-of-range vertex id
    conn[1, 11], conn[2, 11] = conn[2, 11], conn[1, 11]  # inverted cell
    counts = fem.fem_check_mesh(to_dev(case.mesh.coords, torch.float64), to_dev(conn, torch.int32)).cpu().numpy()
    assert counts[0] == 1
    assert counts[1] == 1
    assert counts[3] == 1


def test_deterministic_and_stream(lap3d):
    c, d = device_arrays(lap3d, "mixed")
    r1 = residual(c, d, "mixed").clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r2 = residual(c, d, "mixed", stream=s)
    s.synchronize()
    assert torch.equal(r1, r2)


def test_argument_errors(lap2d):
    c, d = device_arrays(lap2d, "fp64")
    with pytest.raises(ValueError):
        fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"].float(), d["K"], c.rule.points, c.rule.weights,
                                    prec="fp64")
    with pytest.raises(fem.FemError):
        fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points + 1.0, c.rule.weights,
                                    prec="fp64")


@pytest.mark.parametrize("offset", [1e3, -7.5e4])
def test_mixed_form_far_from_origin(offset):
    """The mesh moved far from the origin: the Jacobian columns x_j - x_0 are 6.4e4 to 4.8e6
    times smaller than the coordinates. The mixed form differences the float64 coordinates
    exactly (float32 hi/lo splits) and stays within its tolerance; the float32 ablation, which
    rounds the coordinates first, loses the columns."""
    base = workloads.laplacian_cube_case(6 * 8 ** 3)
    mesh = workloads.Mesh(3, base.mesh.coords + offset, base.mesh.conn)
    case = workloads.Case("laplacian", mesh, base.rule, base.u, K=base.K)
    c, d = device_arrays(case, "mixed")
    ref = oracle.residual_for(c)
    r = residual(c, d, "mixed")
    torch.cuda.synchronize()
    assert rel_err(r, ref) <= TOL["mixed"]
    c32, d32 = device_arrays(case, "fp32")
    r32 = residual(c32, d32, "fp32")
    torch.cuda.synchronize()
    # the ablation's columns are float32 roundings of large numbers: ten times past the
    # mixed form's tolerance already at 1e3
    assert rel_err(r32, ref) > 10 * TOL["mixed"]

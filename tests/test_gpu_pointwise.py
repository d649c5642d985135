"""User pointwise physics compiled at run time (fem_integrate_pointwise; Sec. 5: f0 and f1
given as source text and inlined into the kernel): the two built-in physics written as
strings against the built-in kernels and the oracle, the nonlinear coefficient
kappa(u, x) grad u of Sec. 2 and a reaction + source term against the oracle's pinned
pointwise routine, in float64 and the mixed form, at ragged and full sizes; the compiled
kernels are cached (repeat calls bitwise identical), a source that does not compile
returns the compiler's message, and mesh errors reach fem_device_error."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, rel_err, to_dev

pytestmark = pytest.mark.gpu

LAPLACIAN = "for (int i = 0; i < DIM; ++i) f1[i] = a[0] * grad_u[i];"
LAME = """T tr = T(0);
for (int k = 0; k < DIM; ++k) tr += grad_u[k * DIM + k];
for (int k = 0; k < DIM; ++k)
    for (int i = 0; i < DIM; ++i)
        f1[k * DIM + i] = a[1] * (grad_u[k * DIM + i] + grad_u[i * DIM + k]) + (k == i ? a[0] * tr : T(0));"""
# kappa(u, x) = (p0 + p1 u + p2 u^2)(1 + p3 s(x)), s = x_0 + 2 x_1 (+ 3 x_2): the oracle's "nonlinear"
P_NL = (1.3, -0.7, 0.45, 0.35)
NONLINEAR = """T s = T(0);
for (int i = 0; i < DIM; ++i) s += T(i + 1) * x[i];
const T kappa = (T(%r) + T(%r) * u[0] + T(%r) * u[0] * u[0]) * (T(1) + T(%r) * s);
for (int i = 0; i < DIM; ++i) f1[i] = kappa * grad_u[i];""" % P_NL
P_RE = (0.6, 0.0, 0.0, 0.0)
REACTION_F0 = "f0[0] = a[0] * u[0] + T(%r);" % P_RE[0]
REACTION_F1 = "for (int i = 0; i < DIM; ++i) f1[i] = a[1] * grad_u[i];"


def _dev_case(case, prec):
    c = case if prec == "fp64" else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    return c, to_dev(c.mesh.coords, torch.float64), to_dev(c.mesh.conn, torch.int32), dt


def _lap_case(dim, n):
    return workloads.laplacian_square_case(n) if dim == 2 else workloads.laplacian_cube_case(n)


@pytest.mark.parametrize("dim,n", [(2, 24), (3, 6 * 9 ** 3), (3, 5001)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_laplacian_as_string(dim, n, prec):
    c, coords, conn, dt = _dev_case(_lap_case(dim, n), prec)
    q = c.rule
    u, K = to_dev(c.u, dt), to_dev(c.K, dt)
    r = fem.fem_integrate_pointwise(coords, conn, u, K[None].contiguous(), q.points, q.weights, f1=LAPLACIAN,
                                    prec=prec)
    builtin = fem.fem_integrate_laplacian(coords, conn, u, K, q.points, q.weights, prec=prec)
    ref = oracle.residual_for(c)
    assert rel_err(r, ref) <= TOL[prec]
    # the built-in kernel collapses the quadrature sum (exact algebra for P1); this one
    # evaluates it point by point: equal up to rounding
    assert rel_err(r, builtin.double().cpu().numpy()) <= (1e-13 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_elasticity_as_string(dim, prec):
    c, coords, conn, dt = _dev_case(workloads.elasticity_case(dim, 3001 if dim == 2 else 4099), prec)
    q = c.rule
    u, lam, mu = to_dev(c.u, dt), to_dev(c.lam, dt), to_dev(c.mu, dt)
    r = fem.fem_integrate_pointwise(coords, conn, u, torch.stack([lam, mu]), q.points, q.weights, f1=LAME, prec=prec)
    builtin = fem.fem_integrate_elasticity(coords, conn, u, lam, mu, q.points, q.weights, prec=prec)
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]
    assert rel_err(r, builtin.double().cpu().numpy()) <= (1e-13 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("dim,n", [(2, 40), (3, 6 * 10 ** 3), (3, 1572864)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonlinear_kappa_against_oracle(dim, n, prec):
    c, coords, conn, dt = _dev_case(_lap_case(dim, n), prec)
    q = c.rule
    r = fem.fem_integrate_pointwise(coords, conn, to_dev(c.u, dt), None, q.points, q.weights, f1=NONLINEAR,
                                    prec=prec)
    ref = oracle.pointwise("nonlinear", c.mesh.coords, c.mesh.conn, c.u, None, q.points, q.weights, params=P_NL)
    assert rel_err(r, ref) <= TOL[prec]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reaction_f0_and_f1_against_oracle(dim, prec):
    c, coords, conn, dt = _dev_case(_lap_case(dim, 30 if dim == 2 else 3001), prec)
    q = c.rule
    rng = np.random.default_rng(9)
    coef = np.stack([rng.uniform(0.5, 2.0, c.K.shape), c.K])
    if prec != "fp64":
        coef = coef.astype(np.float32).astype(np.float64)
    r = fem.fem_integrate_pointwise(coords, conn, to_dev(c.u, dt), to_dev(coef, dt), q.points, q.weights,
                                    f0=REACTION_F0, f1=REACTION_F1, prec=prec)
    ref = oracle.pointwise("reaction", c.mesh.coords, c.mesh.conn, c.u, coef, q.points, q.weights, params=P_RE)
    assert rel_err(r, ref) <= TOL[prec]


def test_cache_repeat_bitwise_and_compile_only():
    c, coords, conn, dt = _dev_case(_lap_case(3, 6 * 6 ** 3), "mixed")
    q = c.rule
    u = to_dev(c.u, dt)
    r1 = fem.fem_integrate_pointwise(coords, conn, u, None, q.points, q.weights, f1=NONLINEAR)
    r2 = fem.fem_integrate_pointwise(coords, conn, u, None, q.points, q.weights, f1=NONLINEAR)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2)
    # an empty mesh compiles (and caches) without launching
    empty = torch.zeros((4, 0), dtype=torch.int32, device="cuda")
    out = fem.fem_integrate_pointwise(coords, empty, u, None, q.points, q.weights, f1=LAPLACIAN.replace("a[0]", "T(2)"))
    assert out.shape == (4, 0)


def test_compile_error_is_reported():
    c, coords, conn, dt = _dev_case(_lap_case(3, 6 * 2 ** 3), "fp64")
    q = c.rule
    with pytest.raises(fem.FemError) as ei:
        fem.fem_integrate_pointwise(coords, conn, to_dev(c.u, dt), None, q.points, q.weights,
                                    f1="f1[0] = undefined_name;", prec="fp64")
    assert ei.value.status == -1 and "undefined_name" in str(ei.value)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bad_mesh_reported(prec):
    case = _lap_case(3, 6 * 5 ** 3)
    c, coords, conn, dt = _dev_case(case, prec)
    q = c.rule
    bad = c.mesh.conn.copy()
    bad[2, 7] = bad[1, 7]  # repeated vertex
    assert fem.fem_device_error() == 0
    fem.fem_integrate_pointwise(coords, to_dev(bad, torch.int32), to_dev(c.u, dt), None, q.points, q.weights,
                                f1=NONLINEAR, prec=prec)
    assert fem.fem_device_error() == -5
    bad = c.mesh.conn.copy()
    bad[0, 3] = c.n_verts + 10  # out-of-range id
    fem.fem_integrate_pointwise(coords, to_dev(bad, torch.int32), to_dev(c.u, dt), None, q.points, q.weights,
                                f1=NONLINEAR, prec=prec)
    assert fem.fem_device_error() == -5
    assert fem.fem_device_error() == 0

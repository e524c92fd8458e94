"""pk_grad (the reverse pass on the GPU) against the oracle's reverse pass, finite
differences of the GPU forward, identities, and the torch autograd wrapper."""
import cmath
import math

import numpy as np
import pytest

import knotgen as kg
import oracle.grad as og
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "split": 1e-6, "c64": 1e-3}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def sc(s):
    return SC.of(s.mantissa, s.exp2)


def _sliced_plan(ctx, k, q, **kw):
    """A plan sliced into a few (3..243) slices: the widest tensor's limit is lowered
    step by step from the unsliced width until slicing starts."""
    full = pk.Plan(ctx, k, q, **kw).stats()["log2_max_elems"]
    lim = full
    while lim > 1.0:
        lim -= 0.5
        p = pk.Plan(ctx, k, q, max_log2_elems=lim, **kw)
        if p.stats()["n_slices"] > 1:
            assert p.stats()["n_slices"] <= 243
            return p
    raise AssertionError("no sliced plan")


def _compare(knot, q, z, d, dv, prec, weights=None):
    info, edges = knot.info(), knot.edges()
    zo, do = og.dlogz(info["n_v"], edges, q, weights)
    zz = sc(z)
    assert abs(zz.m * 2.0 ** (zz.e - zo.e) - zo.m) <= TOL[prec] * abs(zo.m)
    scale = max(1.0, float(np.max(np.abs(do)))) if do.size else 1.0
    err = float(np.max(np.abs(d - do), initial=0.0)) / scale
    assert err <= TOL[prec], err
    if weights is None:
        dvo = og.dlogv_dt(info["n_v"], edges, q, info["writhe"], info["tau"])
        assert abs(dv - dvo) <= TOL[prec] * max(1.0, abs(dvo))
    return err


def _knots():
    out = [(kg.braid_closure_pd([1, 1, 1], 2), None),
           (kg.kink(kg.braid_closure_pd([1, -2, 1, -2], 3), 0, 1), None)]
    rng = kg.SplitMix64(77)
    base = kg.random_grid_knot(14, 5, True, 15, 30)
    out.append((kg.randomize(base.pd, rng, 6), None))
    for s in range(4):
        gk = kg.random_grid_knot(18, 300 + s, True, 30, 70)
        out.append((gk.pd, gk.outer))
    return out


@pytest.mark.parametrize("prec", ["c128", "split", "c64"])
def test_grad_matches_oracle(ctx, prec):
    worst = 0.0
    for pd, outer in _knots():
        k = pk.Knot.from_pd(ctx, pd, outer=outer)
        for q in (2, 3, 5):
            for stride in (0, 4):
                p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=stride)
                z, v, d, dv = pk.grad(p, prec)
                worst = max(worst, _compare(k, q, z, d, dv, prec))
                zs, vs = pk.evaluate(p, prec)   # the forward alone agrees
                assert abs(sc(z).m * 2.0 ** (sc(z).e - sc(zs).e) - sc(zs).m) <= TOL[prec]
    print(f"[grad {prec}] worst relative error of dlogZ/dT vs the oracle {worst:.2e}")


@pytest.mark.parametrize("prec", ["c128", "split"])
def test_grad_reconfigured_plans_match_oracle(ctx, prec):
    """Gradient plans with subtree reconfiguration (pk_plan_opts.refine) on the GPU: the
    reverse pass over the rebracketed tree against the oracle's adjoints."""
    for pd, outer in _knots()[2:]:
        k = pk.Knot.from_pd(ctx, pd, outer=outer)
        for q in (3, 5):
            p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=4, refine=8)
            z, v, d, dv = pk.grad(p, prec)
            _compare(k, q, z, d, dv, prec)


def test_grad_sliced_and_forced_kernels(ctx):
    for s in range(3):
        gk = kg.random_grid_knot(16, 400 + s, True, 25, 50)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        for flags in (0, pk.FLAG_FORCE_GEMM, pk.FLAG_FORCE_ROWS):
            p = _sliced_plan(ctx, k, 3, grad=True, checkpoint_stride=2, flags=flags)
            for prec in ("c128", "split"):
                z, v, d, dv = pk.grad(p, prec)
                _compare(k, 3, z, d, dv, prec)


def test_strides_agree_and_repeat(ctx):
    """Recomputing from checkpoints gives the same numbers as keeping every
    intermediate; two calls give identical results."""
    gk = kg.random_grid_knot(20, 7, True, 50, 90)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    ref = None
    for stride in (1, 2, 3, 4, 8):
        p = pk.Plan(ctx, k, 3, grad=True, checkpoint_stride=stride)
        z, v, d, dv = pk.grad(p, "c128")
        z2, v2, d2, dv2 = pk.grad(p, "c128")
        assert np.array_equal(d, d2) and dv == dv2
        if ref is None:
            ref = (z, d, dv)
        else:
            assert np.max(np.abs(d - ref[1])) <= 1e-13 * np.max(np.abs(ref[1]))


def _dlog(zp, zm):
    return cmath.log(zp.mantissa / zm.mantissa) + (zp.exp2 - zm.exp2) * math.log(2.0)


def test_grad_matches_gpu_finite_differences(ctx):
    """Central differences (h = 1e-6) of the GPU forward (complex128) along random
    directions of all edge weights, and along single edges' diagonal and off-diagonal."""
    h = 1e-6
    rng = np.random.default_rng(11)
    for s in range(2):
        gk = kg.random_grid_knot(18, 500 + s, True, 30, 60)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        edges = k.edges()
        for q in (3, 5):
            w0 = og.standard_weights(edges, q)
            p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=4)
            _, _, d, _ = pk.grad(p, "c128")
            eye = np.eye(q, dtype=bool)
            jd = np.array([d[e][eye].sum() for e in range(len(edges))])
            jo = np.array([d[e][~eye].sum() if edges[e][0] != edges[e][1] else 0
                           for e in range(len(edges))])
            dirs = [rng.standard_normal((len(edges), 2)) + 1j * rng.standard_normal((len(edges), 2))]
            for e in (0, len(edges) // 2):
                for j in (0, 1):
                    dd = np.zeros((len(edges), 2), dtype=complex)
                    dd[e, j] = 1.0
                    dirs.append(dd)
            fp = pk.Plan(ctx, k, q, weights=w0)
            for dd in dirs:
                lin = (dd[:, 0] * jd).sum() + (dd[:, 1] * jo).sum()
                fp.set_weights([(a + h * x, b + h * y) for (a, b), (x, y) in zip(w0, dd)])
                zp, _ = pk.evaluate(fp, "c128")
                fp.set_weights([(a - h * x, b - h * y) for (a, b), (x, y) in zip(w0, dd)])
                zm, _ = pk.evaluate(fp, "c128")
                fd = _dlog(zp, zm) / (2 * h)
                assert abs(fd - lin) <= 1e-6 * max(1.0, abs(lin)), (q, fd, lin)


def test_identities_on_gpu(ctx):
    """Linearity in each clause matrix and the colour-permutation symmetry: for every
    edge the joint distribution T_e * dlogZ/dT_e sums to 1 with uniform marginals 1/q."""
    gk = kg.random_grid_knot(22, 21, True, 80, 120)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    edges = k.edges()
    for q in (3, 5):
        w = og.standard_weights(edges, q)
        p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=4)
        for prec in ("c128", "split"):
            _, _, d, _ = pk.grad(p, prec)
            for e, ((u, v, _), (dg, off)) in enumerate(zip(edges, w)):
                if u == v:
                    assert abs(np.trace(d[e]) * dg - 1) < 10 * TOL[prec]
                    continue
                T = np.full((q, q), off, dtype=complex)
                T[np.diag_indices(q)] = dg
                P = T * d[e]
                assert np.allclose(P.sum(axis=0), 1 / q, atol=10 * TOL[prec])
                assert np.allclose(P.sum(axis=1), 1 / q, atol=10 * TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "split"])
def test_grad_workload_300_crossings(ctx, prec):
    """The 300-crossing knot (L=53, seed 7) at q=3 with checkpoints every 4th tree level,
    against the oracle's reverse pass and dV/dt against GPU finite differences of V(t)."""
    (gk,) = kg.knot_suite("grad")
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    assert k.info()["n_c"] == 300
    p = pk.Plan(ctx, k, 3, grad=True, checkpoint_stride=4)
    z, v, d, dv = pk.grad(p, prec)
    err = _compare(k, 3, z, d, dv, prec)
    print(f"[grad workload {prec}] dlogZ/dT max relative error {err:.2e}")
    if prec == "c128":
        info, edges = k.info(), k.edges()
        t, h = og.t_of_q(3), 1e-6
        fp = pk.Plan(ctx, k, 3, weights=og.jones_weights(edges, 3, t))

        def vat(tt):
            fp.set_weights(og.jones_weights(edges, 3, tt))
            zz, _ = pk.evaluate(fp, "c128")
            a = og.prefactor_at(tt, info["n_v"], info["writhe"], info["tau"])
            return pk.Scaled((a.m * zz.mantissa).real, (a.m * zz.mantissa).imag, a.e + zz.exp2)

        fd = _dlog(vat(t + h), vat(t - h)) / (2 * h)
        assert abs(fd - dv) <= 1e-6 * max(1.0, abs(dv)), (fd, dv)


def test_torch_autograd(ctx):
    """log Z through torch.autograd: the weight gradient is the conjugate of the
    holomorphic derivative (PyTorch's convention), and dlogV/dt by the chain rule through
    weights(t) and A(t) equals pk_grad's."""
    import torch
    gk = kg.random_grid_knot(18, 610, True, 30, 60)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    info, edges = k.info(), k.edges()
    q = 3
    p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=4)
    _, _, d, dv = pk.grad(p, "c128")
    w = torch.tensor(og.standard_weights(edges, q), dtype=torch.complex128, requires_grad=True)
    lz = pk.log_z(p, w, "c128")
    (g,) = torch.autograd.grad(lz, w, grad_outputs=torch.ones_like(lz))
    eye = np.eye(q, dtype=bool)
    for e, (u, v, _) in enumerate(edges):
        assert abs(complex(g[e, 0]).conjugate() - d[e][eye].sum()) < 1e-10
        if u != v:
            assert abs(complex(g[e, 1]).conjugate() - d[e][~eye].sum()) < 1e-10
    t = torch.tensor(og.t_of_q(q), dtype=torch.complex128, requires_grad=True)
    eps = torch.tensor([float(e[2]) for e in edges], dtype=torch.float64)
    wt = torch.stack([-(t ** (-eps)), torch.ones_like(eps, dtype=torch.complex128)], dim=1)
    kk = (3 * info["writhe"] + info["tau"] + 2 * info["n_v"] + 2) // 4
    logv = pk.log_z(p, wt, "c128") + kk * torch.log(t) - (info["n_v"] + 1) * torch.log(t + 1)
    (gt,) = torch.autograd.grad(logv, t, grad_outputs=torch.ones_like(logv))
    assert abs(complex(gt).conjugate() - dv) < 1e-10 * max(1.0, abs(dv))

"""The reverse-mode gradient (spmc_grad and its autograd Function) against
central differences on the same Philox streams and against the CPU oracle's
forward-mode tangent.  The walks do not depend on the parameters (common random
numbers), so the estimator is a smooth function of them."""
import numpy as np
import pytest

from tests.common import oracle_spec, oracle_u0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _workload(batch=2, M=512):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w5(M=M, K=2, batch=batch, n_space=5, degree=3, n_intervals=2, T=0.5, n_coef=3)
    wl.kappa = 0.05
    wl.n_ref = 8
    for b, inst in enumerate(wl.instances):
        inst.f_scale = 0.8 + 0.3 * b
    return wl


def _loss_and_z(plan, flat):
    z = plan.final_values(flat)
    return 0.5 * float((z * z).sum()), z


def _solve(api, wl, precision, scales, coefs):
    from paper_2608_22190_b300 import _lib as L
    plan = api.Plan.from_workload(wl, precision=precision)
    for b, inst in enumerate(wl.instances):
        plan.set_problem(b, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, float(scales[b]), inst.ex_kind,
                         inst.ex_beta, np.ascontiguousarray(coefs[b].T).ravel(), L.U0_PHI_COEF, coefs[b].shape[0])
    flat = plan.solve()
    return plan, flat


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import api as A
    return A


@pytest.mark.parametrize("precision,h,rtol", [(0, 1e-5, 1e-6), (1, 1e-5, 1e-5)])
def test_grad_matches_central_differences(api, precision, h, rtol):
    """Central differences of the FP64 solve on the same Philox streams (a smooth
    function of the parameters: the walks do not depend on them).  The mixed
    path's adjoint (FP32 walks and basis values, FP64 accumulation) is compared
    with the same FP64 differences: it differs from them by FP32 rounding of the
    walk and of the basis (about 1e-7 relative) and by the rare walks whose
    decisions flip between FP32 and FP64, well inside 1e-5.  (Differences of the
    mixed solve itself would carry its FP32 rounding divided by h.)"""
    wl = _workload()
    scales = np.array([i.f_scale for i in wl.instances])
    coefs = np.array([i.u0_coef for i in wl.instances])
    plan, flat = _solve(api, wl, precision, scales, coefs)
    L0, z = _loss_and_z(plan, flat)
    gs, gc = plan.grad(z, n_coef=coefs.shape[1])
    gs = gs.cpu().numpy()
    gc = gc.view(-1, coefs.shape[1], coefs.shape[1]).transpose(1, 2).cpu().numpy()
    plan.close()
    rng = np.random.default_rng(4)
    for b in range(len(scales)):
        def loss_at(ds, dc):
            s2 = scales.copy(); s2[b] += ds
            c2 = coefs.copy(); c2[b] += dc
            p, f = _solve(api, wl, 0, s2, c2)
            v, _ = _loss_and_z(p, f)
            p.close()
            return v
        fd_s = (loss_at(h, 0.0) - loss_at(-h, 0.0)) / (2 * h)
        assert abs(fd_s - gs[b]) <= rtol * max(abs(fd_s), 1e-3), (b, fd_s, gs[b])
        dirc = rng.standard_normal(coefs.shape[1:])
        fd_c = (loss_at(0.0, h * dirc) - loss_at(0.0, -h * dirc)) / (2 * h)
        lin = float((gc[b] * dirc).sum())
        assert abs(fd_c - lin) <= rtol * max(abs(fd_c), 1e-3), (b, fd_c, lin)


def test_grad_matches_oracle_tangent(O, api):
    """Directional derivatives from the GPU adjoint (FP64) against the oracle's
    forward-mode tangent on the same walks."""
    wl = _workload(batch=1)
    inst = wl.instances[0]
    scales = np.array([inst.f_scale])
    coefs = np.array([inst.u0_coef])
    plan, flat = _solve(api, wl, 0, scales, coefs)
    _, z = _loss_and_z(plan, flat)
    gs, gc = plan.grad(z, n_coef=coefs.shape[1])
    nc = coefs.shape[1]
    gc = gc.view(nc, nc).transpose(0, 1).cpu().numpy()
    zc = z.cpu().numpy()[0]
    plan.close()
    spec = oracle_spec(O, wl, inst)
    u0 = oracle_u0(O, wl, inst, spec)
    rng = np.random.default_rng(9)
    dirc = rng.standard_normal((nc, nc))
    ds = 0.37
    tmp = type(inst)(t_breaks=inst.t_breaks, degrees=inst.degrees, u0_kind="phi_coef", u0_coef=dirc)
    du0 = oracle_u0(O, wl, tmp, spec)
    blocks, dblocks = O.solve_tangent(spec, inst.t_breaks, inst.degrees, wl.K, u0, du0, ds)
    zdot = dblocks[-1][-1]
    ref = float(zc @ zdot)
    got = float(gs.cpu().numpy()[0] * ds + (gc * dirc).sum())
    assert abs(got - ref) <= 1e-8 * max(abs(ref), 1e-6), (got, ref)


def test_autograd_function(api):
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300.api import SpmcFunction
    wl = _workload()
    plan = api.Plan.from_workload(wl, precision=L.FP64)
    s = torch.tensor([i.f_scale for i in wl.instances], dtype=torch.float64, requires_grad=True)
    c = torch.tensor(np.array([i.u0_coef for i in wl.instances]), dtype=torch.float64, requires_grad=True)
    z = SpmcFunction.apply(s, c, plan, wl)
    loss = 0.5 * (z * z).sum()
    loss.backward()
    gs, gc = plan.grad(z.detach().to("cuda").contiguous(), n_coef=c.shape[1])
    assert torch.allclose(s.grad, gs.cpu(), rtol=1e-12, atol=1e-14)
    assert torch.allclose(c.grad, gc.view(-1, c.shape[1], c.shape[1]).transpose(1, 2).cpu(), rtol=1e-12, atol=1e-14)
    plan.close()


def test_event_adjoint_matches_cohort_adjoint(api):
    """The adjoint sweep on the event pipeline (the iteration's own events,
    outer-product sums per slice) and on the cohort kernel (per-evaluation
    scatters) compute the same gradient: FP64, to rounding of their different
    summation orders."""
    wl = _workload()
    scales = np.array([i.f_scale for i in wl.instances])
    coefs = np.array([i.u0_coef for i in wl.instances])
    out = {}
    for sweep in ("events", "cohort"):
        from paper_2608_22190_b300 import _lib as L
        plan = api.Plan.from_workload(wl, precision=0)
        plan.set_sweep(sweep)
        for b, inst in enumerate(wl.instances):
            plan.set_problem(b, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, float(scales[b]),
                             inst.ex_kind, inst.ex_beta, np.ascontiguousarray(coefs[b].T).ravel(), L.U0_PHI_COEF,
                             coefs[b].shape[0])
        flat = plan.solve()
        _, z = _loss_and_z(plan, flat)
        gs, gc = plan.grad(z, n_coef=coefs.shape[1])
        out[sweep] = (gs.cpu().numpy(), gc.cpu().numpy())
        plan.close()
    for a, b in zip(out["events"], out["cohort"]):
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max()), np.abs(a - b).max()

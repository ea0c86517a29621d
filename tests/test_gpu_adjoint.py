"""GPU adjoint and velocity gradient through the C ABI: the adjoint
dot-product test (to 1e-5), parity of the gradient with the FP64 oracle's
adjoint-state gradient (itself pinned by central differences), invariance to
the checkpoint count, and the torch.autograd entry."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2010_10248_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_10248_gb300 as tb
    tb.load()
    return tb


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(shape=(34, 37, 45), so=8, nt=90, seed=11):
    h = (10.0, 11.0, 9.0)
    vp = wl.layered_vp(shape, seed, vmin=1800.0, vmax=2800.0, nlayers=4, nblobs=4)
    g = np.random.default_rng(seed + 1)
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    src = g.uniform(0.35, 0.65, size=(2, 3)) * ext
    rec = g.uniform(0.1, 0.9, size=(40, 3)) * ext
    # damping held fixed: per-axis sponge of 6 cells at 3000 m/s
    damp = np.concatenate([oracle.damping_axis(shape[d], 6, h[d], 3000.0) for d in range(3)])
    eta = (damp[:shape[0], None, None] + damp[shape[0]:shape[0] + shape[1]][None, :, None]
           + damp[shape[0] + shape[1]:][None, None, :])
    dt = 0.7 * oracle.cfl_dt_max(so, h, vp.max())
    return h, so, nt, vp, damp.astype(np.float32), eta, src, rec, dt, g


def make_prop(tb, shape, h, so, vp, damp, dt, src, wav, rec):
    import torch
    p = tb.Propagator(shape, h, so)
    p.set_model(torch.from_numpy(vp).cuda(), damp=damp, dt=dt)
    p.set_sources(src, wav)
    p.set_receivers(rec)
    return p


def test_adjoint_dot_product(tb):
    import torch
    h, so, nt, vp, damp, eta, src, rec, dt, g = case()
    q = g.standard_normal((2, nt)).astype(np.float32)
    r = g.standard_normal((nt, len(rec))).astype(np.float32)
    p = make_prop(tb, vp.shape, h, so, vp, damp, dt, src, q, rec)
    d = p.forward(nt, schedule="onestep").cpu().numpy()
    gsrc = torch.empty((2, nt), device="cuda")
    p.adjoint_gradient(nt, torch.from_numpy(r).cuda(), grad_src=gsrc, n_snapshots=7)
    lhs = float(np.sum(d.astype(np.float64) * r))
    rhs = float(np.sum(q.astype(np.float64) * gsrc.cpu().numpy()))
    print(f"dot test: <Fq, r> = {lhs:.9e}, <q, F^T r> = {rhs:.9e}, rel {abs(lhs - rhs) / abs(lhs):.2e}")
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("so", [4, 8])
def test_gradient_matches_oracle(tb, so):
    import torch
    h, _, nt, vp, damp, eta, src, rec, dt, g = case(so=so)
    dt = 0.7 * oracle.cfl_dt_max(so, h, vp.max())
    wav = np.repeat(wl.ricker(35.0, dt, nt, t0=6 * dt)[None, :], 2, axis=0).astype(np.float32)
    r = g.standard_normal((nt, len(rec))).astype(np.float32)
    p = make_prop(tb, vp.shape, h, so, vp, damp, dt, src, wav, rec)
    gvp = torch.empty(vp.shape, device="cuda")
    gsrc = torch.empty((2, nt), device="cuda")
    p.adjoint_gradient(nt, torch.from_numpy(r).cuda(), grad_vp=gvp, grad_src=gsrc, n_snapshots=9)
    gsrc_o, gvp_o = oracle.acoustic_adjoint(vp.shape, h, so, dt, nt, vp.astype(np.float64), r.astype(np.float64),
                                            eta=eta, src_xyz=src, src_wav=wav.astype(np.float64), rec_xyz=rec)
    e_g, e_s = rel_l2(gvp.cpu().numpy(), gvp_o), rel_l2(gsrc.cpu().numpy(), gsrc_o)
    print(f"so{so}: grad_vp rel-L2 {e_g:.2e}, grad_src rel-L2 {e_s:.2e}")
    assert e_g <= 1e-4 and e_s <= 1e-4


def test_gradient_independent_of_checkpoints(tb):
    """Recomputation is deterministic: every checkpoint count gives the same
    gradient bit for bit."""
    import torch
    h, so, nt, vp, damp, eta, src, rec, dt, g = case(nt=50)
    wav = np.repeat(wl.ricker(35.0, dt, nt, t0=6 * dt)[None, :], 2, axis=0).astype(np.float32)
    r = torch.from_numpy(g.standard_normal((nt, len(rec))).astype(np.float32)).cuda()
    p = make_prop(tb, vp.shape, h, so, vp, damp, dt, src, wav, rec)
    outs = []
    for ns in (1, 4, 7, 50):
        gvp = torch.empty(vp.shape, device="cuda")
        p.adjoint_gradient(nt, r, grad_vp=gvp, n_snapshots=ns)
        outs.append(gvp.cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_autograd_function(tb):
    import torch
    h, so, nt, vp, damp, eta, src, rec, dt, g = case(nt=40)
    wav = np.repeat(wl.ricker(35.0, dt, nt, t0=6 * dt)[None, :], 2, axis=0).astype(np.float32)
    p = tb.Propagator(vp.shape, h, so)
    v = torch.from_numpy(vp).cuda().requires_grad_(True)
    d_obs = torch.from_numpy(g.standard_normal((nt, len(rec))).astype(np.float32)).cuda() * 1e-9
    tr = tb.AcousticTraces.apply(v, p, src, wav, rec, nt, dt, damp, 8)
    loss = 0.5 * ((tr - d_obs) ** 2).sum()
    loss.backward()
    # the same gradient straight through the C ABI with residual tr - d_obs
    gvp = torch.empty(vp.shape, device="cuda")
    p.adjoint_gradient(nt, (tr - d_obs).detach(), grad_vp=gvp, n_snapshots=8)
    np.testing.assert_array_equal(v.grad.cpu().numpy(), gvp.cpu().numpy())
    assert float(v.grad.abs().max()) > 0


@pytest.mark.parametrize("S", [1, 3, 12])
def test_binomial_schedule_equals_segments(tb, S):
    """The binomial schedule (exactly S stored states) recomputes the same
    forward states by the same one-step sweeps as the segment scheme: the
    gradients in vp and in the wavelets are bit-identical; the forward-step
    count is the planner's, and the scratch holds 2 S + 3 wavefields beside
    the adjoint's own buffers, whatever nt is."""
    import torch
    h, so, nt, vp, damp, eta, src, rec, dt, g = case(nt=61)
    wav = np.repeat(wl.ricker(35.0, dt, nt, t0=6 * dt)[None, :], 2, axis=0).astype(np.float32)
    r = torch.from_numpy(g.standard_normal((nt, len(rec))).astype(np.float32)).cuda()
    p = make_prop(tb, vp.shape, h, so, vp, damp, dt, src, wav, rec)
    res = {}
    for mode in ("segments", "binomial"):
        gvp = torch.empty(vp.shape, device="cuda")
        gsrc = torch.empty((2, nt), device="cuda")
        p.adjoint_gradient(nt, r, grad_vp=gvp, grad_src=gsrc, n_snapshots=S, checkpointing=mode)
        res[mode] = (gvp.cpu().numpy(), gsrc.cpu().numpy(), p.adjoint_stats())
    np.testing.assert_array_equal(res["binomial"][0], res["segments"][0])
    np.testing.assert_array_equal(res["binomial"][1], res["segments"][1])
    assert float(np.abs(res["binomial"][0]).max()) > 0
    _, fsteps = tb.tb_plan_checkpoints(nt, S)
    assert res["binomial"][2][0] == fsteps
    assert res["segments"][2][0] == 2 * nt
    n2p = (vp.shape[2] + 3) // 4 * 4
    field = 4 * vp.shape[0] * vp.shape[1] * n2p
    states = (2 * S + 3) * field
    own = 2 * field + 8 * vp.shape[0] * vp.shape[1] * n2p        # mu pair, FP64 sum
    tables = res["binomial"][2][1] - states - own
    assert 0 <= tables < field, (res["binomial"][2][1], states, own)

"""The learned initial guess on the GPU: the BF16 tensor-core network against
the FP64 oracle (forward and gradient), training with the GPU's own kernels,
and the guess inside the solver (same converged answer, fewer iterations once
trained, plain fallback).

Tolerances: the GPU rounds weights and every hidden activation to BF16
(relative 2^-9) and accumulates in FP32.  The oracle is evaluated with the
same BF16-rounded weights (the parameters the kernels actually multiply), so
what remains is the rounding of three hidden layers and of the BF16 gradient
operands: 2e-2 of the output scale for the forward pass, 5e-2 relative (2-norm
per layer) for the gradient.
"""
import numpy as np
import pytest

import oracle.cnn as OC

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
torch = pytest.importorskip("torch")

# (offset, size, is_weight) of every parameter block
_BLOCKS = []
_o = 0
for _ci, _co, _ in OC.LAYERS:
    _BLOCKS.append((_o, _co * 3 * _ci, True))
    _o += _co * 3 * _ci
    _BLOCKS.append((_o, _co, False))
    _o += _co


def bf16_weights(params):
    """The parameters as the kernels multiply them: weights rounded to BF16, biases FP32."""
    p = np.asarray(params, dtype=np.float32).astype(np.float64)
    out = p.copy()
    for o, n, w in _BLOCKS:
        if w:
            out[o:o + n] = torch.tensor(p[o:o + n]).to(torch.bfloat16).double().numpy()
    return out


def make_batch(nxs, pitch, seed, garbage=100.0):
    """BF16 features [nb, pitch, 16]; cells at or beyond a member's count hold garbage
    (the network must treat them as zero padding)."""
    rng = np.random.default_rng(seed)
    nb = len(nxs)
    f = rng.normal(0.0, 1.0, size=(nb, pitch, N.NH_CNN_IN))
    for b, n in enumerate(nxs):
        f[b, n:] = garbage
    ft = torch.tensor(f, dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    nxd = torch.tensor(nxs, dtype=torch.int32, device="cuda")
    return ft, nxd


def oracle_forward(ft, nxs, params):
    f = ft.float().cpu().double().numpy()
    return [OC.forward_member(f[b, :n], params) for b, n in enumerate(nxs)]


@pytest.mark.parametrize("nxs,pitch", [([1000, 257, 130, 8], 1024), ([120, 121, 239, 240, 241], 256)])
def test_forward_matches_oracle(nxs, pitch):
    params = OC.init_params(3)
    params[1536:1568] = 0.1          # non-zero biases
    params[9312:] = -0.05
    pt = torch.tensor(params, dtype=torch.float32, device="cuda")
    ft, nxd = make_batch(nxs, pitch, seed=11)
    y = N.nh_cnn_forward(ft, nxd, pt, out_scale=2.0)
    torch.cuda.synchronize()
    y = y.cpu().double().numpy()
    ref = oracle_forward(ft, nxs, bf16_weights(params))
    scale = max(np.max(np.abs(r)) for r in ref)
    for b, n in enumerate(nxs):
        err = np.max(np.abs(y[b, :n] - 2.0 * ref[b]))
        assert err <= 2e-2 * 2.0 * scale, (b, err, scale)
        assert np.all(y[b, n:] == 0.0)          # cells outside the member are not written
    # against the full-precision parameters the BF16 weight rounding adds a little
    ref_full = oracle_forward(ft, nxs, params)
    err_full = max(np.max(np.abs(y[b, :n] - 2.0 * ref_full[b])) for b, n in enumerate(nxs))
    assert err_full <= 4e-2 * 2.0 * scale


def test_forward_full_size_sampled():
    """64 members x 50000 cells (the slide batch's size), members 0 and 63 checked."""
    nxs = [50000] * 64
    pitch = 50176
    params = OC.init_params(5)
    pt = torch.tensor(params, dtype=torch.float32, device="cuda")
    ft, nxd = make_batch(nxs, pitch, seed=12, garbage=0.0)
    y = N.nh_cnn_forward(ft, nxd, pt)
    torch.cuda.synchronize()
    f = ft[[0, 63]].float().cpu().double().numpy()
    yw = y[[0, 63]].cpu().double().numpy()
    pw = bf16_weights(params)
    for k in range(2):
        ref = OC.forward_member(f[k, :50000], pw)
        assert np.max(np.abs(yw[k, :50000] - ref)) <= 2e-2 * np.max(np.abs(ref))


def test_gradient_matches_oracle():
    nxs, pitch = [1000, 257, 130, 8], 1024
    params = OC.init_params(7)
    params[4640:4672] = 0.05
    pt = torch.tensor(params, dtype=torch.float32, device="cuda")
    ft, nxd = make_batch(nxs, pitch, seed=13)
    rng = np.random.default_rng(14)
    tgt = rng.normal(0.0, 1.0, size=(len(nxs), pitch))
    msk = (rng.random((len(nxs), pitch)) < 0.6).astype(np.uint8)
    for b, n in enumerate(nxs):
        msk[b, n:] = 1                      # outside the member: must be ignored anyway
    tt = torch.tensor(tgt, dtype=torch.float32, device="cuda")
    mt = torch.tensor(msk, device="cuda")
    # the mask count the oracle normalises by: counted cells inside the members
    inside = np.zeros_like(msk)
    for b, n in enumerate(nxs):
        inside[b, :n] = msk[b, :n]
    mt_in = torch.tensor(inside, device="cuda")
    grad = torch.zeros(N.NH_CNN_PARAMS, dtype=torch.float32, device="cuda")
    loss = N.nh_cnn_loss_grad(ft, nxd, pt, tt, mt, grad)
    g_out = grad.clone()
    # mask entries outside the members change nothing
    loss_in = N.nh_cnn_loss_grad(ft, nxd, pt, tt, mt_in, grad)
    assert loss == pytest.approx(loss_in, rel=1e-12)
    g = grad.cpu().double().numpy()
    f = ft.float().cpu().double().numpy()
    t32 = tt.cpu().double().numpy()
    xs = [f[b, :n] for b, n in enumerate(nxs)]
    ts = [t32[b, :n] for b, n in enumerate(nxs)]
    ms = [inside[b, :n] for b, n in enumerate(nxs)]
    ref_loss, ref_g = OC.loss_and_grad(xs, bf16_weights(params), ts, ms)
    assert abs(loss_in - ref_loss) <= 2e-2 * ref_loss
    # FP32 atomics accumulate in a run-dependent order: entries agree to the
    # rounding of the largest contributions
    assert torch.allclose(g_out, grad, rtol=1e-4, atol=1e-5 * float(grad.abs().max()))
    for o, n, w in _BLOCKS:
        d = np.linalg.norm(g[o:o + n] - ref_g[o:o + n])
        assert d <= 5e-2 * np.linalg.norm(ref_g[o:o + n]) + 1e-7, (o, n, d, np.linalg.norm(ref_g[o:o + n]))


def test_training_reduces_loss():
    """Adam with the GPU's own forward/backward kernels on a learnable task
    (target = a fixed linear stencil of two feature channels)."""
    nxs, pitch = [4096] * 8, 4096
    ft, nxd = make_batch(nxs, pitch, seed=21, garbage=0.0)
    f = ft.float()
    tgt = 0.5 * torch.roll(f[:, :, 0], 1, dims=1) - 0.25 * f[:, :, 1] + 0.3 * torch.roll(f[:, :, 2], -1, dims=1)
    tgt[:, 0] = 0.0
    tgt[:, -1] = 0.0
    msk = torch.ones((len(nxs), pitch), dtype=torch.uint8, device="cuda")
    msk[:, 0] = 0
    msk[:, -1] = 0
    params = torch.tensor(OC.init_params(1), dtype=torch.float32, device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    ws = N.CnnWorkspace(len(nxs), pitch)
    tgt = tgt.contiguous()
    first = None
    for step in range(1, 301):
        loss = N.nh_cnn_loss_grad(ft, nxd, params, tgt, msk, grad, ws)
        first = loss if first is None else first
        N.nh_cnn_adam(params, grad, m, v, step, 3e-3)
    final = N.nh_cnn_loss_grad(ft, nxd, params, tgt, msk, grad, ws)
    assert np.isfinite(final)
    assert final < 0.05 * first, (first, final)


# ------------------------------------------------------------ in the solver

from paper_2505_17025_gb300 import guess_train as GT   # noqa: E402


def _slide_grid(wl, guess=N.NH_GUESS_PREV, crit=N.NH_CRIT_GLOBAL, knh=1e-3):
    G = N.grid_from_workload(wl)
    G.set_criterion(crit, knh, 1, False)
    G.cnn_attach()
    G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, guess)
    return G


@pytest.fixture(scope="module")
def slide_wl():
    from paper_2505_17025_gb300 import workloads as W
    return W.slide_1d(n_members=4, nx=20000)


def _run_steps(G, dt, n):
    iters = 0
    for _ in range(n):
        st, info = G.step(dt)
        iters += info["iters"]
    return iters


def _psi(G, dt, nx):
    h, _, _, p = G.get_state()
    return np.asarray(p) * np.asarray(h) * (dt / 1000.0)     # nh_get_state: p = rho psi / (dt h)


def test_harvest_consistent(slide_wl):
    """The harvested target is what the quadratic extrapolation misses, in
    units of S2, on the marked cells with three previous solutions."""
    G = _slide_grid(slide_wl)
    G.cnn_record(True)
    dt = slide_wl.dt
    _run_steps(G, dt, 3)
    psis = [_psi(G, dt, 20000)]
    for _ in range(3):
        G.step(dt)
        psis.append(_psi(G, dt, 20000))
    feat, tgt, msk, S2 = G.cnn_harvest()
    assert S2 > 0.0
    m = msk.cpu().numpy()[:, :20000].astype(bool)
    assert m.sum() > 0.9 * m.size    # global criterion: every cell has its history
    t = tgt.cpu().numpy()[:, :20000]
    # psi^{n+1} - psi^n - d1 - D2 = third difference
    expect = (psis[3] - 3.0 * psis[2] + 3.0 * psis[1] - psis[0]) / S2
    scale = max(np.max(np.abs(expect[m])), np.max(np.abs(psis[3])) / S2 * 1e-12)
    assert np.max(np.abs(t[m] - expect[m])) <= 1e-3 * scale
    f = feat.float().cpu().numpy()
    assert np.all(f[:, :20000, 2][m] == 1.0)      # channel 2: marked for the step
    assert np.all(f[:, :20000, 5][m] == 1.0)      # channel 5: second difference defined
    assert np.all(f[:, 20000:] == 0.0)
    assert np.max(np.abs(f[:, :20000, 0])) == pytest.approx(1.0, abs=1e-2)   # d1 / S1
    assert np.max(np.abs(f[:, :20000, 4])) == pytest.approx(1.0, abs=1e-2)   # D2 / S2


@pytest.mark.parametrize("precond", [N.NH_PRECOND_NONE, N.NH_PRECOND_LINE])
def test_learned_guess_same_answer_and_fewer_iterations(precond):
    """Train on pairs the plain method generates, then continue the run from
    the learned start: same converged state; without a preconditioner (where
    the start decides the iteration count) at least 20 % fewer Krylov
    iterations than the plain warm start, with the line preconditioner (an
    almost exact solve) no more than 2 % more."""
    from paper_2505_17025_gb300 import workloads as W
    wl = W.slide_1d(n_members=2, nx=5000)
    dt = wl.dt
    n_train, n_eval = 60, 30

    def grid():
        G = _slide_grid(wl)
        G.set_preconditioner(precond)
        return G

    A = grid()
    samples = GT.collect(A, dt, n_train)
    params, losses = GT.train(samples, steps=400)
    assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5]), (losses[:5], losses[-20:])
    B = grid()
    _run_steps(B, dt, n_train)
    assert np.array_equal(np.asarray(A.get_state()[0]), np.asarray(B.get_state()[0]))
    A.cnn_set_params(params)
    A.cnn_record(False)
    A.set_solver(N.NH_SOLVER_AUTO, 1e-12, 200000, N.NH_GUESS_CNN)
    B.set_solver(N.NH_SOLVER_AUTO, 1e-12, 200000, N.NH_GUESS_PREV)
    it_cnn = _run_steps(A, dt, n_eval)
    it_prev = _run_steps(B, dt, n_eval)
    hA, huA, _, _ = A.get_state()
    hB, huB, _, _ = B.get_state()
    amp = wl.amplitude
    assert np.max(np.abs(np.asarray(hA) - np.asarray(hB))) <= 1e-9 * amp
    assert np.max(np.abs(np.asarray(huA) - np.asarray(huB))) <= 1e-9 * amp * np.sqrt(9.81)
    ch = A.cnn_choices()
    print(f"precond {precond}: iterations over {n_eval} steps: learned start {it_cnn}, "
          f"previous pressure {it_prev}; starts {ch}")
    assert sum(ch.values()) == 2 * n_eval
    if precond == N.NH_PRECOND_NONE:
        assert it_cnn <= 0.8 * it_prev, (it_cnn, it_prev)
    else:
        assert it_cnn <= 1.02 * it_prev, (it_cnn, it_prev)


def test_network_learns_adaptive_target(slide_wl):
    """On the adaptive slide (|eta/d| > 1e-4) the trained network predicts
    held-out targets better than the extrapolation alone (output 0)."""
    dt = slide_wl.dt
    G = _slide_grid(slide_wl, crit=N.NH_CRIT_ETA_D, knh=1e-4)
    _run_steps(G, dt, 200)
    train = GT.collect(G, dt, 120)
    held = GT.collect(G, dt, 40)
    assert len(train) > 60 and len(held) > 20
    params, _ = GT.train(train, steps=400)
    num = den = 0.0
    for f, t, m, nxd in held:
        y = N.nh_cnn_forward(f.contiguous(), nxd, params)
        mm = m.float()
        num += float(((y - t) ** 2 * mm).sum())
        den += float((t ** 2 * mm).sum())
    rel = (num / den) ** 0.5
    print(f"held-out relative error of the trained correction: {rel:.3f} (zero correction: 1)")
    assert rel < 0.9


def test_untrained_and_nonfinite_networks(slide_wl):
    """A random network and a network that outputs NaN converge to the answer
    of the plain warm start; the NaN network's start is never chosen."""
    dt = slide_wl.dt
    runs = {}
    for name in ("prev", "random", "nan"):
        G = _slide_grid(slide_wl)
        if name != "prev":
            p = torch.tensor(OC.init_params(9), dtype=torch.float32, device="cuda")
            if name == "nan":
                p[:] = float("nan")
            G.cnn_set_params(p)
            G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_CNN)
        it = _run_steps(G, dt, 30)
        runs[name] = (G.get_state(), it, G.cnn_choices() if name != "prev" else None)
    amp = slide_wl.amplitude
    s_prev = runs["prev"][0]
    for name in ("random", "nan"):
        s, it, ch = runs[name]
        assert it > 0
        assert np.max(np.abs(np.asarray(s[0]) - np.asarray(s_prev[0]))) <= 1e-9 * amp
        assert np.max(np.abs(np.asarray(s[1]) - np.asarray(s_prev[1]))) <= 1e-9 * amp * np.sqrt(9.81)
    assert runs["nan"][2]["network"] == 0


def test_learned_guess_graph_equals_steps(slide_wl):
    dt = slide_wl.dt
    p = GT.init_params(4, last_gain=1.0)
    out = []
    for graphs in (False, True):
        G = _slide_grid(slide_wl, crit=N.NH_CRIT_ETA_D, knh=1e-5)
        G.cnn_set_params(p)
        G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_CNN)
        G.set_run_mode(graphs)
        st, info = G.run(dt, 30)
        out.append((G.get_state(), info["iters_total"], G.cnn_choices()))
    (s0, i0, c0), (s1, i1, c1) = out
    assert i0 > 0
    for k in range(3):
        a, b = np.asarray(s0[k]), np.asarray(s1[k])
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(a)))
    assert i0 == i1
    assert c0 == c1

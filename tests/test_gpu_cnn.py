"""Learned warm start: the GPU network against the FP64 reference
(oracle/cnn.py) on the same BF16 operands, layer by layer (forward) and for
the gradient of the mean squared error (backward), bound 1e-5 relative;
Adam against its textbook update; training on pairs the solver records;
and what the trained network gains as a warm start (V-cycles), with the
multigrid residual deciding whether a prediction is kept and the same
tolerance met."""
import numpy as np
import pytest

import synth
from helpers import EPS0, Q, gpu_mesh
from oracle import cnn

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def pkg():
    import paper_1708_08434_gb300 as p
    return p


def params(seed=1):
    p = synth.cnn_initial_params().astype(np.float64)
    rng = np.random.default_rng(seed)
    W1, b1, W2, b2, W3, b3 = cnn.unpack(p)
    b1[:] = rng.uniform(-0.2, 0.2, 16)
    b2[:] = rng.uniform(-0.2, 0.2, 16)
    b3[:] = rng.uniform(-0.2, 0.2, 1)
    return cnn.pack(W1, b1, W2, b2, W3, b3).astype(np.float32)


def effective(p):
    """Parameters as the GPU uses them: BF16 weights, FP32 biases."""
    W1, b1, W2, b2, W3, b3 = cnn.unpack(np.asarray(p, np.float64))
    return cnn.pack(cnn.bf16(W1), b1, cnn.bf16(W2), b2, cnn.bf16(W3), b3)


def inputs(n, seed=2):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (n, 1000, 2)).astype(np.float32)


def oracle_x(xb):
    """[1000][2] position-major -> [2][10][10][10] ([z][y][x]), BF16."""
    return cnn.bf16(xb).reshape(10, 10, 10, 2).transpose(3, 0, 1, 2)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def test_forward_layerwise_against_fp64():
    p = params()
    net = pkg().Network(64, 64)
    net.set_params(p)
    x = inputs(5)
    out, acts = net.forward(x, acts=True)
    W1, b1, W2, b2, W3, b3 = cnn.unpack(effective(p))
    for b in range(5):
        X = oracle_x(x[b])
        z1, a1, z2, a2 = (acts[b, i].reshape(16, 8, 8, 8).astype(np.float64) for i in range(4))
        assert rel(z1, cnn.conv(X, W1, b1, True)) <= TOL
        assert np.array_equal(a1, cnn.bf16(np.maximum(z1, 0)))
        assert rel(z2, cnn.conv(a1, W2, b2, False)) <= TOL
        assert np.array_equal(a2, cnn.bf16(np.maximum(z2, 0)))
        ref = cnn.conv(a2, W3[None], b3, False)[0]
        assert rel(out[b].reshape(8, 8, 8).astype(np.float64), ref) <= TOL
        assert (a1 > 0).mean() > 0.2 and (a2 > 0).mean() > 0.2   # ReLUs are exercised


def test_forward_end_to_end_against_oracle():
    """The oracle's own forward pass (FP64 arithmetic, hidden activations
    rounded to BF16 after each ReLU) against the GPU output on the same BF16
    inputs and weights.  The two agree to FP32 accumulation error except
    where that error moves a hidden pre-activation across a BF16 rounding
    boundary: the activation then differs by one BF16 step, 2^-8 of its
    value.  Bound: max |gpu - oracle| <= 2^-8 max |oracle| over each box,
    and no more than 1% of the outputs off by more than 1e-5 relative."""
    p = params(11)
    net = pkg().Network(64, 64)
    net.set_params(p)
    n = 8
    x = inputs(n, 12)
    out = net.forward(x)
    pe = effective(p)
    worst, off = 0.0, 0
    for b in range(n):
        ref = cnn.forward(pe, oracle_x(x[b]), round_acts=True)[-1]
        got = out[b].reshape(8, 8, 8).astype(np.float64)
        worst = max(worst, rel(got, ref))
        off += int((np.abs(got - ref) > 1e-5 * np.abs(ref).max()).sum())
    print("end-to-end forward: max rel %.3e, outputs beyond 1e-5: %d of %d" % (worst, off, n * 512))
    assert worst <= 2.0 ** -8
    assert off <= 0.01 * n * 512


def test_gradient_against_fp64_backprop():
    p = params(3)
    net = pkg().Network(64, 64)
    net.set_params(p)
    n = 6
    x = inputs(n, 4)
    t = np.random.default_rng(5).standard_normal((n, 512)).astype(np.float32) * 0.3
    out, acts = net.forward(x, acts=True)
    g, loss = net.gradient(x, t)
    pe = effective(p)
    scale = 1.0 / (n * 512)
    ref = np.zeros(cnn.N_PARAMS)
    ref_loss = 0.0
    for b in range(n):
        X = oracle_x(x[b])
        a1 = acts[b, 1].reshape(16, 8, 8, 8).astype(np.float64)
        a2 = acts[b, 3].reshape(16, 8, 8, 8).astype(np.float64)
        o = out[b].reshape(8, 8, 8).astype(np.float64)
        tt = t[b].reshape(8, 8, 8).astype(np.float64)
        ref += cnn.backward(pe, X, a1, a2, o, tt, scale)
        ref_loss += scale * np.sum((o - tt) ** 2)
    assert loss == pytest.approx(ref_loss, rel=TOL)
    gr = cnn.unpack(ref)
    gg = cnn.unpack(g.astype(np.float64))
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), gg, gr):
        assert rel(a, b) <= TOL, name


def test_gradient_accumulates_over_the_boxes_of_a_block():
    """A gradient pass runs one block per SM at most, so with more boxes than
    SMs a block takes several boxes, and the layer-2 weight gradient sums
    over them in tensor memory.  The mean squared error over 50 copies of
    the same 6 boxes has the gradient of the 6 boxes alone: compared with
    the FP64 backpropagation of the 6 boxes at the same bound."""
    p = params(13)
    rep = 50
    net = pkg().Network(6 * rep, 64)
    net.set_params(p)
    x = inputs(6, 14)
    t = np.random.default_rng(15).standard_normal((6, 512)).astype(np.float32) * 0.3
    out, acts = net.forward(x, acts=True)
    g, loss = net.gradient(np.tile(x, (rep, 1, 1)), np.tile(t, (rep, 1)))
    pe = effective(p)
    ref = np.zeros(cnn.N_PARAMS)
    for b in range(6):
        ref += cnn.backward(pe, oracle_x(x[b]), acts[b, 1].reshape(16, 8, 8, 8).astype(np.float64),
                            acts[b, 3].reshape(16, 8, 8, 8).astype(np.float64),
                            out[b].reshape(8, 8, 8).astype(np.float64),
                            t[b].reshape(8, 8, 8).astype(np.float64), 1.0 / (6 * 512))
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), cnn.unpack(g.astype(np.float64)),
                          cnn.unpack(ref)):
        assert rel(a, b) <= TOL, name


def test_samples_loaded_explicitly_train_and_time():
    """Explicit samples replace the recorded ones: training on them lowers
    the loss, and the kernel timing runs over them."""
    n = 256
    net = pkg().Network(n, n)
    net.set_params(params(16))
    rng = np.random.default_rng(17)
    net.load_samples(inputs(n, 18), (0.3 * rng.standard_normal((n, 512))).astype(np.float32))
    assert net.stats()["samples"] == n
    first = net.train(1, 64, 1e-3)
    last = net.train(20, 64, 1e-3)
    assert np.isfinite(last) and last < first
    for kind in (0, 1):
        us, fl, tf = net.kernel_bench(kind, n, 2)
        assert us > 0 and fl > 0 and tf > 0


def test_adam_against_textbook_update():
    p = params(6)
    net = pkg().Network(64, 64)
    net.set_params(p)
    rng = np.random.default_rng(7)
    w, m, v = p.astype(np.float64), np.zeros(cnn.N_PARAMS), np.zeros(cnn.N_PARAMS)
    for step in (1, 2, 3):
        g = rng.standard_normal(cnn.N_PARAMS).astype(np.float32)
        net.adam_step(g, 1e-3)
        w, m, v = cnn.adam(w, m, v, g.astype(np.float64), step, 1e-3)
        assert rel(net.get_params().astype(np.float64), w) <= 1e-6


def streamer_run(net_mode=None, net=None, steps=6, per_solve=256):
    """A few Heun steps of the small streamer; returns the solver and the
    V-cycles of every warm-started solve."""
    dom, st = synth.workload("streamer_small")
    g = gpu_mesh(dom, st)
    t = g.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    p = pkg()
    g.upload(p.NE, ne)
    g.upload(p.NI, ni)
    g.set_table(synth.coefficient_table())
    g.charge_rhs(Q, EPS0)
    g.fmg(1e-8, 40)
    g.compute_field()
    if net is not None:
        net.attach(g, net_mode, per_solve=per_solve)
    dt = g.dt_limit(Q, EPS0)
    cycles = []
    for _ in range(steps):
        rc, dtn, c1, c2 = g.advance(dt, Q, EPS0, 1e-8, 40)
        assert rc == 0
        cycles += [c1, c2]
        dt = dtn
    g.dt_next = dt
    return g, cycles


def test_training_on_recorded_solves_reduces_loss():
    net = pkg().Network(4096, 1024)
    net.set_params(synth.cnn_initial_params())
    g, cyc = streamer_run(1, net, steps=4)
    n = net.stats()["samples"]
    assert n >= 8 * 16
    first = net.train(1, 32, 1e-3)
    last = net.train(40, 32, 1e-3)
    print("samples %d loss first epoch %.4e after 41 epochs %.4e" % (n, first, last))
    assert np.isfinite(last) and last < 0.9 * first


def test_learned_warm_start_gain():
    """Train on the pairs recorded during the first steps of a run, then
    measure what the network gained on pairs it never saw (recorded during
    the following steps, with the trained weights frozen: Adam with a zero
    learning rate only evaluates the loss): its mean squared error must be
    below that of the zero prediction (the plain warm start, loss = mean of
    t^2).  Measured: 57.1 against 58.5, a gain of 2.5% -- most unseen
    targets sit at the clip of the per-box scaling, which a per-box network
    with a 7^3 receptive field cannot predict.  In the solver the residual
    test decides: a prediction is kept only when it lowers the relative
    residual, so the learned run never takes more V-cycles than the plain
    one; on this mesh the predictions are not kept."""
    p_ = pkg()
    net = p_.Network(8192, 1024)
    net.set_params(synth.cnn_initial_params())
    streamer_run(1, net, steps=6)
    net.train(60, 32, 1e-3)
    trained = net.get_params()
    # held-out pairs: steps 7-10 of the same run, recorded by a second
    # network that holds the trained weights
    held = p_.Network(8192, 1024)
    held.set_params(trained)
    g_rec, _ = streamer_run(None, None, steps=6)
    held.attach(g_rec, 1, per_solve=256)
    dt = g_rec.dt_next
    for _ in range(4):
        rc, dt, c1, c2 = g_rec.advance(dt, Q, EPS0, 1e-8, 40)
        assert rc == 0
    held.attach(g_rec, 0)
    assert held.stats()["samples"] >= 8 * 64
    loss_trained = held.train(1, 64, 0.0)
    held.set_params(np.zeros_like(trained))
    loss_zero = held.train(1, 64, 0.0)
    print("held-out loss: trained %.4e, zero prediction %.4e" % (loss_trained, loss_zero))
    assert np.isfinite(loss_trained) and loss_trained < loss_zero
    # the solver with predictions: same tolerance met, never more V-cycles
    g_plain, c_plain = streamer_run(None, None, steps=10)
    g_pred, _ = streamer_run(None, None, steps=6)
    net.attach(g_pred, 2, per_solve=1024, taper=True)
    dt = g_pred.dt_next
    c_pred = []
    for _ in range(4):
        rc, dtn, c1, c2 = g_pred.advance(dt, Q, EPS0, 1e-8, 40)
        assert rc == 0
        c_pred += [c1, c2]
        dt = dtn
    s = net.stats()
    plain_eval = c_plain[12:]
    print("V-cycles per warm-started solve, plain %s learned %s; predictions kept %d/%d"
          % (plain_eval, c_pred, s["kept"], s["predictions"]))
    assert s["predictions"] == 8
    assert sum(c_pred) <= sum(plain_eval)

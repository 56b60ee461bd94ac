"""GPU tests of the learned subgrid-stress closure against the FP64 reference (oracle/sgs_mlp.py).

Tolerances: FP64 spectral helpers agree with the reference to ~1e-13 (held to
1e-10); the BF16 network is compared with the reference evaluated on the same
BF16-rounded inputs, weights and activations, so only FP32-versus-FP64
accumulation order differs (held to 1e-2 of the output scale, 3e-2 relative
for gradient blocks).
"""

import numpy as np
import pytest

from oracle import sgs_mlp as sg
from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def _sgs():
    from paper_1602_03638_gb300 import sgs

    return sgs


def _rand_spec(N, seed, dtype=torch.complex128):
    return inputs.isotropic_spectral(N, seed=seed, k0=N / 5.0).to(dtype).cuda()


def test_filter_gradient_products_force_match_reference():
    sgs = _sgs()
    fine = _rand_spec(32, 1)
    got = sgs.spectral_filter(fine, 16, "f64").cpu().numpy()
    ref = sg.filter_truncate(fine.cpu().numpy(), 16)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    uh = _rand_spec(16, 2)
    g9 = sgs.spectral_gradient(uh, "f64").cpu().numpy()
    K = sn.wavenumbers(16)
    for i in range(3):
        for j in range(3):
            np.testing.assert_allclose(g9[3 * i + j], 1j * K[j] * uh[i].cpu().numpy(), atol=1e-12)
    u = torch.randn(3, 16, 16, 16, dtype=torch.float64, device="cuda")
    p6 = sgs.pointwise_products(u, "f64").cpu().numpy()
    un = u.cpu().numpy()
    for c, (i, j) in enumerate(sg.TAU_INDEX):
        np.testing.assert_allclose(p6[c], un[i] * un[j], rtol=0, atol=1e-14)
    tau = np.random.default_rng(3).standard_normal((6, 16, 16, 16))
    th = torch.from_numpy(sn.forward(tau)).cuda()
    f = sgs.stress_force(th, "f64").cpu().numpy()
    fr = sg.stress_force(tau)
    assert np.abs(f - fr).max() < 1e-10 * np.abs(fr).max()


def test_training_data_matches_reference():
    sgs = _sgs()
    Nf, Nc = 32, 16
    uh = inputs.isotropic_spectral(Nf, seed=7, k0=4.0)
    with Solver(Nf, 0.01, 0.01, "f64") as fine, Solver(Nc, 0.01, 0.01, "f64") as coarse:
        fine.set_state_spectral(uh.numpy())
        X, T, ubh = sgs.filtered_training_data(fine, coarse)
        X, T = X.cpu().numpy(), T.cpu().numpy()
    tau_ref, ubh_ref = sg.sgs_stress(uh.numpy(), Nc)
    A_ref = sg.velocity_gradients(ubh_ref)
    # features and targets are FP32 arrays built from FP64 fields
    assert np.abs(X[:9] - A_ref.reshape(9, -1)).max() < 1e-6 * np.abs(A_ref).max()
    assert np.allclose(X[9], 2 * np.pi / Nc)
    assert np.abs(T - tau_ref.reshape(6, -1)).max() < 1e-6 * np.abs(tau_ref).max()
    assert np.abs(ubh.cpu().numpy() - ubh_ref).max() < 1e-12 * np.abs(ubh_ref).max()


def _params_with_norm(seed, X):
    p = sg.init_params(seed)
    rng = np.random.default_rng(seed)
    p["b1"] = rng.normal(size=64) * 0.1
    p["b2"] = rng.normal(size=64) * 0.1
    p["b3"] = rng.normal(size=6) * 0.1
    p["in_shift"] = X.mean(0)
    p["in_scale"] = 1.0 / X.std(0)
    p["out_scale"] = rng.uniform(0.5, 2.0, size=6)
    p["out_shift"] = rng.normal(size=6)
    return p


def test_network_forward_matches_bf16_reference():
    sgs = _sgs()
    rng = np.random.default_rng(5)
    P = 1000
    X = rng.normal(size=(P, 10)) * rng.uniform(0.1, 3.0, size=10)
    p = _params_with_norm(1, X)
    net = sgs.MLP(sg.flatten(p).astype(np.float32))
    pv = sg.unflatten(net.get_params().astype(np.float64))  # FP32-rounded parameters
    tau = net.forward(torch.from_numpy(X.T.astype(np.float32)).cuda().contiguous()).cpu().numpy().T
    ref = sg.forward(pv, X.astype(np.float32).astype(np.float64), round_bf16=True)["tau"]
    assert np.abs(tau - ref).max() < 1e-2 * np.abs(ref).max()
    net.close()


def test_tensor_core_forward_agrees_with_the_training_kernel():
    """Inference (tcgen05, 128-point tiles in TMEM) against the training kernel's own forward
    pass (wmma): the loss of the inferred stress equals the loss the training kernel reports."""
    sgs = _sgs()
    rng = np.random.default_rng(15)
    P = 3 * 128 + 77
    X = rng.normal(size=(P, 10))
    Tt = rng.normal(size=(P, 6))
    p = _params_with_norm(7, X)
    net = sgs.MLP(sg.flatten(p).astype(np.float32))
    pv = sg.unflatten(net.get_params().astype(np.float64))
    Xd = torch.from_numpy(X.T.astype(np.float32)).cuda().contiguous()
    Td = torch.from_numpy(Tt.T.astype(np.float32)).cuda().contiguous()
    tau = net.forward(Xd).cpu().numpy().astype(np.float64).T
    y = (tau - pv["out_shift"]) / pv["out_scale"]
    tn = (Tt.astype(np.float32).astype(np.float64) - pv["out_shift"]) / pv["out_scale"]
    loss_tc = float(np.mean((y - tn) ** 2))
    loss_train, _ = net.loss_grad(Xd, Td)
    assert abs(loss_tc - loss_train) < 1e-4 * loss_train, (loss_tc, loss_train)
    net.close()


def test_network_gradient_matches_bf16_reference():
    sgs = _sgs()
    rng = np.random.default_rng(6)
    P = 777  # not a multiple of the 16-point tile
    X = rng.normal(size=(P, 10))
    Tt = rng.normal(size=(P, 6))
    p = _params_with_norm(2, X)
    net = sgs.MLP(sg.flatten(p).astype(np.float32))
    pv = sg.unflatten(net.get_params().astype(np.float64))
    loss, g = net.loss_grad(torch.from_numpy(X.T.astype(np.float32)).cuda().contiguous(),
                            torch.from_numpy(Tt.T.astype(np.float32)).cuda().contiguous())
    lref, gref = sg.loss_and_grads(pv, X.astype(np.float32).astype(np.float64), Tt.astype(np.float32).astype(np.float64),
                                   round_bf16=True)
    assert abs(loss - lref) < 1e-3 * lref
    gv = sg.unflatten(g.astype(np.float64))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.linalg.norm(gv[name] - gref[name]) / np.linalg.norm(gref[name])
        assert err < 3e-2, (name, err)
    assert np.all(gv["in_shift"] == 0) and np.all(gv["out_scale"] == 0)
    net.close()


def test_adam_update_matches_reference():
    """Three dns_mlp_train_step calls against the FP64 Adam of the reference fed with the same
    FP32 gradient (dns_mlp_loss_grad on the same batch just before each step): the parameter
    trajectories agree to FP32 rounding of an update of size ~lr."""
    sgs = _sgs()
    rng = np.random.default_rng(11)
    P = 2048
    X = rng.normal(size=(P, 10))
    Tt = rng.normal(size=(P, 6))
    p = _params_with_norm(4, X)
    net = sgs.MLP(sg.flatten(p).astype(np.float32))
    Xd = torch.from_numpy(X.T.astype(np.float32)).cuda().contiguous()
    Td = torch.from_numpy(Tt.T.astype(np.float32)).cuda().contiguous()
    lr = 1e-2
    start = sg.unflatten(net.get_params().astype(np.float64))
    ref, st = start, sg.adam_init(start)
    for _ in range(3):
        _, g = net.loss_grad(Xd, Td)
        net.train_step(Xd, Td, lr, want_loss=False)
        got = sg.unflatten(net.get_params().astype(np.float64))
        ref, st = sg.adam_step(ref, sg.unflatten(g.astype(np.float64)), st, lr)
        for name in sg.PARAM_ORDER:
            err = np.abs(got[name] - ref[name]).max()
            assert err < 1e-4 * lr + 2e-7 * np.abs(ref[name]).max(), (st["t"], name, err)
    moved = np.abs(sg.flatten(got) - sg.flatten(start))
    assert np.median(moved[20:5274]) > 0.5 * lr  # Adam moves most weights by ~lr per step
    for name in ("in_shift", "in_scale", "out_scale", "out_shift"):
        assert np.array_equal(got[name], start[name])
    net.close()


def test_network_training_reduces_loss():
    sgs = _sgs()
    rng = np.random.default_rng(8)
    P = 4096
    X = rng.normal(size=(10, P)).astype(np.float32)
    Y = np.stack([np.tanh(X[0] * X[1]), X[2] ** 2 - 1, np.sin(X[3]), X[4] * 0.5, X[5] - X[6], X[7] * X[8]]).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    net = sgs.MLP(seed=3)
    net.set_params(sgs.with_normalisation(net.get_params(), Xd, Yd))
    hist = net.fit(Xd, Yd, iters=400, lr=3e-3, batch=4096, log_every=399)
    assert hist[-1][1] < 0.2 * hist[0][1], hist
    net.close()


def test_forced_rhs_matches_reference():
    N, nu = 16, 0.02
    uh = inputs.isotropic_spectral(N, seed=9, k0=3.0).numpy()
    f = inputs.isotropic_spectral(N, seed=10, k0=5.0).numpy() * 3.0
    with Solver(N, nu, 0.01, "f64") as s:
        s.set_state_spectral(uh)
        s.set_option("use_graph", 1)
        from paper_1602_03638_gb300 import _lib
        import ctypes

        _lib.check(_lib.lib().dns_set_forcing(s.handle, ctypes.c_void_p(f.ctypes.data), 0), "dns_set_forcing")
        got = s.rhs()
        # stepping with the force matches the reference RK4 with the same force
        s.step(3)
        stepped = s.get_state_spectral()
    g = sn.Grid(N)
    ref = sg.rhs_forced(uh, g, nu, sn.zero_nyquist(f))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    cur = uh
    fz = sn.zero_nyquist(f)
    for _ in range(3):
        u0, u1 = cur.copy(), cur.copy()
        for st in range(4):
            d = sg.rhs_forced(cur, g, nu, fz)
            if st < 3:
                cur = u0 + sn.RK4_B[st] * 0.01 * d
            u1 = u1 + sn.RK4_A[st] * 0.01 * d
        cur = u1
    assert np.linalg.norm(stepped - cur) / np.linalg.norm(cur) < 1e-12


def _closure_net(seed, N):
    """A network with random weights and biases, normalised on the features of a random field."""
    sgs = _sgs()
    rng = np.random.default_rng(seed)
    p = sg.init_params(seed)
    p["b1"] = rng.normal(size=64) * 0.1
    p["b2"] = rng.normal(size=64) * 0.1
    p["b3"] = rng.normal(size=6) * 0.1
    net = sgs.MLP(sg.flatten(p).astype(np.float32))
    X = torch.from_numpy(rng.normal(size=(10, N ** 3)).astype(np.float32) * 3.0).cuda()
    T = torch.from_numpy(rng.normal(size=(6, N ** 3)).astype(np.float32) * 0.01).cuda()
    net.set_normalisation(X, T)
    return net


def test_normalisation_kernel_matches_mean_and_unbiased_std():
    sgs = _sgs()
    rng = np.random.default_rng(12)
    P = 5000
    X = rng.normal(size=(10, P)) * rng.uniform(0.1, 5.0, size=(10, 1)) + rng.normal(size=(10, 1))
    X[9] = 0.25  # a constant feature keeps scale 1
    T = rng.normal(size=(6, P)) * 0.02 + 0.3
    net = sgs.MLP(seed=0)
    before = sg.unflatten(net.get_params().astype(np.float64))
    net.set_normalisation(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda())
    got = sg.unflatten(net.get_params().astype(np.float64))
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(got["in_shift"], X32.mean(1), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(got["in_scale"][:9], 1.0 / X32[:9].std(1, ddof=1), rtol=1e-6)
    assert got["in_scale"][9] == 1.0
    np.testing.assert_allclose(got["out_scale"], T32.std(1, ddof=1), rtol=1e-6)
    np.testing.assert_allclose(got["out_shift"], T32.mean(1), rtol=1e-6)
    for k in sg.TRAINABLE:
        assert np.array_equal(got[k], before[k])
    net.close()


def test_in_step_closure_equals_the_composed_calls():
    """dns_set_closure (features, network, force and forcing inside the step graph) against the
    same closure composed from the library's separate calls before every step: bit for bit."""
    sgs = _sgs()
    N, nu, dt, steps = 32, 0.01, 0.005, 3
    uh = inputs.isotropic_spectral(N, seed=21, k0=4.0).numpy().astype(np.complex64)
    net = _closure_net(3, N)
    with Solver(N, nu, dt, "f32") as a, Solver(N, nu, dt, "f32") as b:
        sgs.on_torch_stream(a, b)
        a.set_state_spectral(uh)
        b.set_state_spectral(uh)
        a.set_closure(net)
        a.step(steps)
        for _ in range(steps):
            sgs.set_closure_force(b, net)
            b.step(1)
        ga, gb = a.get_state_spectral(), b.get_state_spectral()
    assert np.abs(ga - uh).max() > 1e-4 * np.abs(uh).max()  # the state moved
    np.testing.assert_array_equal(ga, gb)
    net.close()


def test_in_step_closure_rhs_matches_reference():
    """dns_rhs with the closure attached against the reference: features from the reference's
    velocity gradients, its BF16-rounded network, stress force and forced right-hand side."""
    N, nu = 32, 0.01
    uh = inputs.isotropic_spectral(N, seed=22, k0=4.0).numpy().astype(np.complex64)
    net = _closure_net(4, N)
    with Solver(N, nu, 0.005, "f32") as s:
        s.set_state_spectral(uh)
        s.set_closure(net)
        got = s.rhs()
        s.set_closure(None)
        plain = s.rhs()
    pv = sg.unflatten(net.get_params().astype(np.float64))
    u64 = uh.astype(np.complex128)
    A = sg.velocity_gradients(u64).reshape(9, -1)
    X = np.concatenate([A, np.full((1, N ** 3), 2 * np.pi / N)]).T
    tau = sg.forward(pv, X, round_bf16=True)["tau"].T.reshape(6, N, N, N)
    f = sg.stress_force(tau)
    g = sn.Grid(N)
    ref = sg.rhs_forced(u64, g, nu, f)
    fscale = np.abs(f * g.mask).max()
    assert fscale > 1e-3 * np.abs(ref).max()  # the closure term is not negligible
    assert np.abs(got - ref).max() < 2e-2 * fscale + 1e-5 * np.abs(ref).max()
    # detaching restores the plain right-hand side
    assert np.abs(plain - sn.rhs(u64, g, nu)).max() < 1e-5 * np.abs(ref).max()
    net.close()


def test_trained_closure_beats_the_unmodelled_coarse_run():
    """A-posteriori: 256^3 DNS (this solver) -> box-filtered 32^3 data -> network trained on the
    GPU -> coarse 32^3 runs with and without the closure, compared against the filtered DNS."""
    sgs = _sgs()
    r = sgs.closure_experiment(Nf=256, Nc=32, nu=2e-3, dt_f=2e-3, dt_c=5e-3, t_dev=0.4, t_run=0.8,
                               iters=400, batch=32768, seed=0)
    losses = [l for _, l in r["train_loss"]]
    assert losses[-1] < 0.6 * losses[0]
    rows = r["checkpoints"]
    # the closure supplies the missing subgrid dissipation ...
    assert np.mean([x["model"]["dissipation_err"] for x in rows]) < 0.7 * np.mean([x["no_model"]["dissipation_err"] for x in rows])
    # ... and keeps the resolved spectrum closer to the filtered DNS
    assert np.mean([x["model"]["spectrum_err"] for x in rows]) < np.mean([x["no_model"]["spectrum_err"] for x in rows])

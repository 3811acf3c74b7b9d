"""The learned warm start: the library's FP32 network kernels against the FP64
oracle network, and the start it gives the LM solve against the
nearest-training-point start."""

import numpy as np
import pytest

from oracle import mlp as om
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ARCH = (2, 128, 3, 48)  # mu -> 3 hidden layers of 128 -> 48 outputs


def _data(seed, n, n_in, n_out):
    x = W.normal(seed, 1, n * n_in).reshape(n, n_in)
    t = W.normal(seed, 2, n * n_out).reshape(n, n_out)
    return x, t


def _params(seed, arch):
    p = np.zeros(om.n_params(*arch))
    k = 0
    g = W.normal(seed, 3, p.size)
    for i, o in om.layer_sizes(*arch):
        p[k:k + i * o] = g[k:k + i * o] / np.sqrt(i)
        k += i * o
        p[k:k + o] = 0.1 * g[k:k + o]
        k += o
    return p.astype(np.float32).astype(np.float64)  # exactly representable in the network's FP32 storage


def test_parameter_count_and_roundtrip():
    net = ift.MLP(*ARCH, seed=1)
    assert net.n_params == om.n_params(*ARCH) == 2 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 48 + 48
    p = _params(5, ARCH)
    net.set_params(p)
    np.testing.assert_array_equal(net.get_params(), p)
    # seeded initialisation: b = 0, W with standard deviation about 1/sqrt(in)
    net2 = ift.MLP(*ARCH, seed=1)
    q = om.unpack(net2.get_params(), *ARCH)
    assert all(np.all(b == 0) for _, b in q)
    assert abs(np.std(q[1][0]) * np.sqrt(128) - 1) < 0.05
    np.testing.assert_array_equal(ift.MLP(*ARCH, seed=1).get_params(), net2.get_params())


def test_forward_matches_oracle():
    net = ift.MLP(*ARCH, seed=0)
    p = _params(7, ARCH)
    net.set_params(p)
    x, _ = _data(8, 37, 2, 48)  # a ragged row count
    y = net.predict(x)  # untrained network: no standardisation
    ref, _ = om.forward(p, x, *ARCH)
    assert np.max(np.abs(y - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("rows", [37, 300, 4096])
def test_bf16_tensor_core_forward_matches_oracle(rows):
    # The tensor-core path rounds the operands of every width-input product to BF16
    # (unit roundoff 2^-9) and accumulates in FP32; through the three products the
    # outputs carry a relative error of order 1e-2, the stated BF16 tolerance.
    net = ift.MLP(*ARCH, seed=0)
    p = _params(7, ARCH)
    net.set_params(p)
    x, _ = _data(9, rows, 2, 48)  # 37 and 300 rows leave a partial 128-row tile
    y16 = net.predict_bf16(x)
    ref, _ = om.forward(p, x, *ARCH)
    assert np.linalg.norm(y16 - ref) <= 2e-2 * np.linalg.norm(ref)
    assert np.max(np.abs(y16 - ref)) <= 5e-2 * np.max(np.abs(ref))
    # it is the BF16 path: the FP32 network is far closer to the FP64 reference
    y32 = net.predict(x)
    assert np.max(np.abs(y32 - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(y16 - y32)) > 1e-4 * np.max(np.abs(ref))
    # the same inputs give the same outputs on a second call
    np.testing.assert_array_equal(net.predict_bf16(x), y16)


def test_bf16_forward_after_training_and_shape_limits():
    mus = W.mu_box_samples(80, 1, 256)
    t = np.stack([mus[:, 0] * (2 + k) + np.cos(30 * mus[:, 1]) for k in range(16)], axis=1)
    net = ift.MLP(2, 64, 2, 16, seed=81)
    net.train(mus, t, epochs=100, batch=64, lr=3e-3, seed=82)
    q = W.mu_box_samples(83, 1, 200)
    y32, y16 = net.predict(q), net.predict_bf16(q)  # standardisation applied and undone alike
    assert np.linalg.norm(y16 - y32) <= 2e-2 * np.linalg.norm(y32)
    with pytest.raises(ift.IFTError) as ei:
        ift.MLP(2, 20, 2, 4, seed=1).predict_bf16(q)  # width not a multiple of 16
    assert ei.value.status == -7


def test_gradient_matches_oracle():
    net = ift.MLP(*ARCH, seed=0)
    p = _params(9, ARCH)
    net.set_params(p)
    x, t = _data(10, 16, 2, 48)
    loss, g = net.loss_grad(x, t)
    rl, rg = om.loss_and_grad(p, x, t, *ARCH)
    assert abs(loss - rl) <= 1e-5 * rl
    assert np.linalg.norm(g - rg) <= 1e-4 * np.linalg.norm(rg)
    # layer by layer, so a wrong block cannot hide behind a large one
    k = 0
    for i, o in om.layer_sizes(*ARCH):
        for n in (i * o, o):
            assert np.linalg.norm(g[k:k + n] - rg[k:k + n]) <= 1e-4 * max(np.linalg.norm(rg[k:k + n]), 1e-12)
            k += n


def test_gradient_against_device_finite_differences():
    # independent of the oracle: central differences of the device loss on the
    # eight largest gradient entries
    arch = (2, 16, 2, 3)
    net = ift.MLP(*arch, seed=0)
    p = _params(11, arch)
    net.set_params(p)
    x, t = _data(12, 64, 2, 3)
    _, g = net.loss_grad(x, t)
    for j in np.argsort(-np.abs(g))[:8]:
        h = 2.0 ** -7
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        net.set_params(pp)
        lp, _ = net.loss_grad(x, t, want_grad=False)
        net.set_params(pm)
        lm, _ = net.loss_grad(x, t, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-2 * abs(g[j]), (j, fd, g[j])
    net.set_params(p)


def test_training_fits_a_smooth_map():
    mus = W.mu_box_samples(20, 1, 512)
    u = (mus - W.MU_BOX_LO) / W.MU_BOX_WIDTH
    t = np.stack([np.sin(2 * u[:, 0] + k * u[:, 1]) * (1 + 0.1 * k) + 3 * k for k in range(6)], axis=1)
    net = ift.MLP(2, 64, 2, 6, seed=3)
    before = np.mean((net.predict(mus) - t) ** 2)
    final = net.train(mus, t, epochs=300, batch=64, lr=3e-3, seed=4)
    assert final < 1e-3
    q = W.mu_box_samples(21, 1, 256)
    uq = (q - W.MU_BOX_LO) / W.MU_BOX_WIDTH
    tq = np.stack([np.sin(2 * uq[:, 0] + k * uq[:, 1]) * (1 + 0.1 * k) + 3 * k for k in range(6)], axis=1)
    after = np.mean((net.predict(q) - tq) ** 2)
    assert after < 1e-3 * before and after < 1e-2


def test_nearest_start_is_the_nearest_point():
    xt = W.mu_box_samples(30, 1, 300)
    yt = W.normal(30, 2, 300 * 5).reshape(300, 5)
    xq = W.mu_box_samples(31, 1, 77)
    scale = 1.0 / W.MU_BOX_WIDTH
    out = ift.nearest_start(xt, yt, xq, scale=scale)
    d = (((xq[:, None, :] - xt[None, :, :]) * scale) ** 2).sum(-1)
    np.testing.assert_array_equal(out, yt[np.argmin(d, axis=1)])
    # exact hits return their own row (distance 0, lowest index on ties)
    np.testing.assert_array_equal(ift.nearest_start(xt, yt, xt[:10]), yt[:10])


def test_errors():
    with pytest.raises(ift.IFTError):
        ift.MLP(0, 8, 1, 1)
    with pytest.raises(ift.IFTError):
        ift.MLP(2, 0, 1, 1)
    net = ift.MLP(2, 8, 1, 1)
    with pytest.raises(ift.IFTError):
        net.train(np.zeros((1, 2)), np.zeros((1, 1)), 1, 1, 1e-3)
    with pytest.raises(ift.IFTError):
        net.train(np.zeros((4, 2)), np.zeros((4, 1)), 1, 4, 0.0)


def _train_and_solve(n, ku, kx, n_train, n_query, width, epochs, rho_set):
    wl = W.euler_workload(n=n, p=2, k_u=ku, k_x=kx, seed=40)
    mu_t = W.mu_box_samples(41, 1, n_train)
    mu_q = W.mu_box_samples(42, 1, n_query)
    # training solutions from the method itself (projected-guess start)
    gen = ift.Context.from_workload(wl, tol=1e-8)
    gen.set_eq_weights_batched([rho_set] * n_train)
    res = gen.solve_rom_batched(mu_t)
    ok = np.array([i["status"] == 0 for i in res["info"]])
    assert ok.mean() > 0.95
    y_t = np.concatenate([res["w"], res["tau"]], axis=1)[ok]
    mu_t = mu_t[ok]
    net = ift.MLP(2, width, 3, ku + kx, seed=43)
    net.train(mu_t, y_t, epochs=epochs, batch=32, lr=2e-3, seed=44)
    starts = {"mlp": net.predict(mu_q), "mlp_bf16": net.predict_bf16(mu_q),
              "nearest": ift.nearest_start(mu_t, y_t, mu_q, scale=1.0 / W.MU_BOX_WIDTH)}
    ctx = ift.Context.from_workload(wl, tol=1e-8, lm_init=ift.INIT_GIVEN)
    ctx.set_eq_weights_batched([rho_set] * n_query)
    ref = ift.Context.from_workload(wl, tol=1e-8)
    ref.set_eq_weights_batched([rho_set] * n_query)
    exact = ref.solve_rom_batched(mu_q)
    z_ref = np.concatenate([exact["w"], exact["tau"]], axis=1)
    out = {}
    for name, s in starts.items():
        r = ctx.solve_rom_batched(mu_q, s[:, :ku], s[:, ku:])
        st = np.array([i["status"] for i in r["info"]])
        it = np.array([i["iters"] + i["init_iters"] for i in r["info"]])
        err = np.linalg.norm(s - z_ref, axis=1) / np.linalg.norm(z_ref, axis=1)
        zf = np.concatenate([r["w"], r["tau"]], axis=1)
        out[name] = dict(status=st, iters=it, start_err=err, final=zf, J=np.array([i["J"] for i in r["info"]]))
    return out, exact


def test_warm_start_beats_nearest_training_point():
    wl_sets = W.euler_workload(n=16, p=2, k_u=10, k_x=2, seed=40)
    rho_set = W.eq_weight_sets(wl_sets, 1, seed=45, lo=120, hi=121)[0]
    out, exact = _train_and_solve(16, 10, 2, 192, 64, 64, 400, rho_set)
    m, m16, nn = out["mlp"], out["mlp_bf16"], out["nearest"]
    # every start converges to the same solutions as the projected-guess start
    for r in (m, m16, nn):
        assert (r["status"] == 0).mean() >= 0.95
    ok = ((m["status"] == 0) & (m16["status"] == 0) & (nn["status"] == 0)
          & np.array([i["status"] == 0 for i in exact["info"]]))
    z_ref = np.concatenate([exact["w"], exact["tau"]], axis=1)
    for r in (m, m16, nn):
        d = np.linalg.norm(r["final"][ok] - z_ref[ok], axis=1) / np.linalg.norm(z_ref[ok], axis=1)
        assert np.max(d) < 1e-5
    # the learned start (FP32 or BF16 network) is closer to the solution and needs
    # fewer LM iterations than the nearest training point
    for r in (m, m16):
        assert np.median(r["start_err"]) < 0.5 * np.median(nn["start_err"])
        assert r["iters"][ok].mean() < nn["iters"][ok].mean()


def test_trained_network_checkpoint_roundtrip(tmp_path):
    from paper_2305_15661_gb300 import checkpoint as ck

    mus = W.mu_box_samples(70, 1, 128)
    t = np.stack([mus[:, 0] * (3 + k) + np.sin(40 * mus[:, 1]) for k in range(4)], axis=1)
    net = ift.MLP(2, 32, 2, 4, seed=71)
    net.train(mus, t, epochs=50, batch=32, lr=3e-3, seed=72)
    wl = W.euler_workload(n=4, p=1, k_u=3, k_x=1, seed=5)
    ck.save_model(str(tmp_path / "m"), wl, mlp=net, train_mu=mus, train_y=t)
    arrays, meta = ck.load(str(tmp_path / "m"))
    net2 = ck.restore_mlp(arrays, meta)
    q = W.mu_box_samples(73, 1, 17)
    np.testing.assert_array_equal(net2.predict(q), net.predict(q))
    np.testing.assert_array_equal(arrays["train_y"], t)

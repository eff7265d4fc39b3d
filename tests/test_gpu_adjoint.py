"""Parity of the CUDA reverse mode with the FP64 oracle: the force VJP kernel
(nb_force_vjp) and the checkpointed fixed-step Hermite trajectory gradient
(nb_traj_forward / nb_traj_backward, and the torch.autograd.Function on top).
"""
import numpy as np
import pytest

import oracle
from synth import plummer
from nbtest import nb  # noqa: F401

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def _ctx(nb, m, x, v, eps, precision, level=0):
    return nb.Context(m, x, v, eps, precision=precision, level_fixed=level, flags=nb.NB_INIT_NO_FORCE)


@pytest.mark.parametrize("n", [2, 7, 300, 1000])
@pytest.mark.parametrize("eps", [1 / 256, 0.0])
def test_force_vjp_fp64_matches_oracle(nb, n, eps):
    m, x, v = plummer(n, 50 + n)
    r = np.random.default_rng(n)
    ab, kb = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    c = _ctx(nb, m, x, v, eps, nb.NB_FP64)
    try:
        got = c.nb_force_vjp(ab, kb)
    finally:
        c.nb_free()
    ref = oracle.force_vjp(m, x, v, eps, ab, kb)
    for g, q in zip(got, ref):
        assert _rel(g, q) < 1e-10


@pytest.mark.parametrize("n", [64, 1000, 4099])
def test_force_vjp_ds_matches_oracle(nb, n):
    m, x, v = plummer(n, 60 + n)
    r = np.random.default_rng(n)
    ab, kb = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    c = _ctx(nb, m, x, v, 1 / 256, nb.NB_DS)
    try:
        got = c.nb_force_vjp(ab, kb)
    finally:
        c.nb_free()
    ref = oracle.force_vjp(m, x, v, 1 / 256, ab, kb)
    for g, q in zip(got, ref):
        assert np.linalg.norm(g - q) <= 2e-5 * np.linalg.norm(q)


def _traj(nb, m, x, v, eps, level, steps, ck, precision, xbT, vbT):
    c = _ctx(nb, m, x, v, eps, precision, level)
    try:
        c.nb_traj_forward(steps, ck)
        st = c.nb_get_state()
        grads = c.nb_traj_backward(xbT, vbT)
        st2 = c.nb_get_state()
        grads2 = c.nb_traj_backward(xbT, vbT)
    finally:
        c.nb_free()
    for key in st:
        assert np.array_equal(st[key], st2[key]), key   # backward leaves the final state
    for g, h in zip(grads, grads2):
        assert np.array_equal(g, h)                     # and can be repeated
    return st, grads


@pytest.mark.parametrize("steps,ck", [(24, 5), (24, 24), (7, 1)])
def test_trajectory_gradient_fp64_matches_oracle(nb, steps, ck):
    n, eps, level = 64, 1 / 64, 7
    m, x, v = plummer(n, 70)
    r = np.random.default_rng(71)
    xbT, vbT = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    st, (xb, vb, mb) = _traj(nb, m, x, v, eps, level, steps, ck, nb.NB_FP64, xbT, vbT)
    xt, vt, oxb, ovb, omb = oracle.traj_vjp(m, x, v, eps, 2.0 ** -level, steps, xbT, vbT)
    assert _rel(st["x"], xt) < 1e-12 and _rel(st["v"], vt) < 1e-12
    assert _rel(xb, oxb) < 1e-9 and _rel(vb, ovb) < 1e-9 and _rel(mb, omb) < 1e-9


def test_trajectory_gradient_ds_matches_oracle(nb):
    n, eps, level, steps = 256, 1 / 256, 8, 32
    m, x, v = plummer(n, 80)
    tgt = plummer(n, 81)[1]
    xt, _ = oracle.traj_final(m, x, v, eps, 2.0 ** -level, steps)
    xbT = 2 * (xt - tgt)
    st, (xb, vb, mb) = _traj(nb, m, x, v, eps, level, steps, 8, nb.NB_DS, xbT, None)
    _, _, oxb, ovb, omb = oracle.traj_vjp(m, x, v, eps, 2.0 ** -level, steps, xbT, np.zeros((n, 3)))
    for g, q in ((xb, oxb), (vb, ovb), (mb, omb)):
        assert np.linalg.norm(g - q) <= 1e-4 * np.linalg.norm(q)


def test_checkpoint_spacing_does_not_change_the_gradient(nb):
    n, eps, level, steps = 200, 1 / 256, 9, 20
    m, x, v = plummer(n, 90)
    r = np.random.default_rng(91)
    xbT, vbT = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    base = None
    for ck in (1, 3, 7, 20):
        _, grads = _traj(nb, m, x, v, eps, level, steps, ck, nb.NB_DS, xbT, vbT)
        if base is None:
            base = grads
        for g, h in zip(grads, base):
            assert np.array_equal(g, h), ck


def test_gradient_matches_gpu_fp64_finite_differences(nb):
    # Directional derivatives of f = <xbar_T, x_T> by central differences of
    # the GPU FP64 trajectory itself.
    n, eps, level, steps = 32, 1 / 64, 6, 10
    m, x, v = plummer(n, 95)
    r = np.random.default_rng(96)
    xbT = r.normal(size=(n, 3))

    def f(mm, xx, vv):
        c = _ctx(nb, mm, xx, vv, eps, nb.NB_FP64, level)
        try:
            c.nb_traj_forward(steps, steps)
            return float(np.sum(xbT * c.nb_get_state()["x"]))
        finally:
            c.nb_free()

    _, (xb, vb, mb) = _traj(nb, m, x, v, eps, level, steps, 4, nb.NB_FP64, xbT, None)
    h = 1e-6
    for _ in range(3):
        dx, dv, dm = r.normal(size=(n, 3)), r.normal(size=(n, 3)), r.normal(size=n) * 1e-3
        fd = (f(m + h * dm, x + h * dx, v + h * dv) - f(m - h * dm, x - h * dx, v - h * dv)) / (2 * h)
        an = np.sum(xb * dx) + np.sum(vb * dv) + np.sum(mb * dm)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_autograd_function_loss_backward(nb, monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_cs_0702135_gb300.autograd import hermite_trajectory
    n, eps, level, steps = 128, 1 / 256, 8, 16
    m, x, v = plummer(n, 97)
    tgt = torch.from_numpy(plummer(n, 98)[1]).cuda()
    x0 = torch.from_numpy(x).cuda().requires_grad_(True)
    v0 = torch.from_numpy(v).cuda().requires_grad_(True)
    mm = torch.from_numpy(m).cuda().requires_grad_(True)
    # the Function must stay on the device: the host-array entry points and
    # host copies of CUDA tensors are unavailable while it runs
    def host_path(*a, **k):
        raise AssertionError("host round trip inside hermite_trajectory")
    with monkeypatch.context() as mp:
        for name in ("nb_init", "nb_get_state", "nb_traj_backward", "nb_set_state"):
            mp.setattr(nb.nb, name, host_path)
        mp.setattr(torch.Tensor, "cpu", host_path)
        mp.setattr(torch.Tensor, "numpy", host_path)
        xT, vT = hermite_trajectory(x0, v0, mm, eps, level, steps, 4, nb.NB_FP64)
        assert xT.is_cuda and vT.is_cuda
        loss = ((xT - tgt) ** 2).sum()
        loss.backward()
    assert x0.grad.is_cuda and mm.grad.is_cuda
    xt, _ = oracle.traj_final(m, x, v, eps, 2.0 ** -level, steps)
    _, _, oxb, ovb, omb = oracle.traj_vjp(m, x, v, eps, 2.0 ** -level, steps,
                                          2 * (xt - tgt.cpu().numpy()), np.zeros((n, 3)))
    assert _rel(x0.grad.cpu().numpy(), oxb) < 1e-9
    assert _rel(v0.grad.cpu().numpy(), ovb) < 1e-9
    assert _rel(mm.grad.cpu().numpy(), omb) < 1e-9
    # the library context is released after the first backward: a second
    # backward through the same trajectory is refused
    x1 = torch.from_numpy(x).cuda().requires_grad_(True)
    xT2, _ = hermite_trajectory(x1, v0.detach(), mm.detach(), eps, level, steps, 4, nb.NB_FP64)
    l2 = (xT2 ** 2).sum()
    l2.backward(retain_graph=True)
    with pytest.raises(RuntimeError):
        l2.backward()


def test_device_init_and_state_match_the_host_entry_points(nb):
    torch = pytest.importorskip("torch")
    n, eps = 700, 1 / 256
    m, x, v = plummer(n, 99)
    a = nb.Context(m, x, v, eps)
    b = nb.Context.from_device(torch.from_numpy(m).cuda(), torch.from_numpy(x).cuda(),
                               torch.from_numpy(v).cuda(), eps)
    try:
        for c in (a, b):
            c.nb_run(1.0 / 16)
        sa = a.nb_get_state()
        d = {k: torch.empty((n, 3), dtype=torch.float64, device="cuda") for k in "xvak"}
        dt = torch.empty(n, dtype=torch.int64, device="cuda")
        dl = torch.empty(n, dtype=torch.int32, device="cuda")
        b.nb_get_state_dev(d["x"], d["v"], d["a"], d["k"], dt, dl)
        torch.cuda.synchronize()
        for k in "xvak":
            assert np.array_equal(d[k].cpu().numpy(), sa[k]), k
        assert np.array_equal(dt.cpu().numpy(), sa["t"]) and np.array_equal(dl.cpu().numpy(), sa["level"])
    finally:
        a.nb_free()
        b.nb_free()
    bad = torch.from_numpy(x).cuda()
    bad[5, 1] = float("nan")
    with pytest.raises(nb.NbError) as ei:
        nb.Context.from_device(torch.from_numpy(m).cuda(), bad, torch.from_numpy(v).cuda(), eps)
    assert ei.value.code == nb.NB_EINVAL
    neg = torch.from_numpy(m).cuda()
    neg[3] = -1.0
    with pytest.raises(nb.NbError):
        nb.Context.from_device(neg, torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), eps)


def test_traj_backward_dev_matches_host(nb):
    torch = pytest.importorskip("torch")
    n, eps = 200, 1 / 256
    m, x, v = plummer(n, 101)
    r = np.random.default_rng(5)
    xb, vb = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    c = _ctx(nb, m, x, v, eps, nb.NB_DS, level=9)
    try:
        c.nb_traj_forward(24, 8)
        host = c.nb_traj_backward(xb, vb)
        out = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
        out.append(torch.empty(n, dtype=torch.float64, device="cuda"))
        c.nb_traj_backward_dev(torch.from_numpy(xb).cuda(), torch.from_numpy(vb).cuda(), *out)
        for g, h in zip(out, host):
            assert np.array_equal(g.cpu().numpy(), h)
        bad = torch.from_numpy(xb).cuda()
        bad[0, 0] = float("inf")
        with pytest.raises(nb.NbError) as ei:
            c.nb_traj_backward_dev(bad, None, *out)
        assert ei.value.code == nb.NB_EINVAL
    finally:
        c.nb_free()

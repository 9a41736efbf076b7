"""GPU parity of the U-Net kernels (forward, gradient, Adam) with oracle/cnn.py,
the learner's features with their definition, and the learned / history
coarse spaces inside topology-optimisation steps."""
import numpy as np
import pytest

import workloads
from oracle import cnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, W, N, CIN, COUT = 32, 24, 2, 3, 4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def net():
    from paper_1501_06211_gb300 import ddel
    code, h = ddel.ddel_cnn_create(CIN, COUT, H, W, N, seed=7)
    assert code == 0
    yield h
    ddel.ddel_cnn_destroy(h)


def params(h):
    from paper_1501_06211_gb300 import ddel
    p = np.zeros(ddel.ddel_cnn_num_params(h), dtype=np.float32)
    assert ddel.ddel_cnn_get_params(h, p, 0) == 0
    return p


def batch(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, CIN, H, W)).astype(np.float32)
    t = rng.standard_normal((N, COUT, H, W)).astype(np.float32)
    return x, t


def test_param_count_and_init(net):
    from paper_1501_06211_gb300 import ddel
    assert ddel.ddel_cnn_num_params(net) == cnn.num_params(CIN, COUT)
    p = params(net).astype(float)
    off = 0
    for (co, ci, k, _) in cnn.layer_shapes(CIN, COUT):
        nw = co * ci * k * k
        a = np.sqrt(6.0 / (ci * k * k))
        w = p[off:off + nw]
        assert np.all(np.abs(w) <= a) and np.std(w) > 0.3 * a  # U(-a, a): std a / sqrt(3)
        assert np.all(p[off + nw:off + nw + co] == 0.0)
        off += nw + co


def test_forward_matches_oracle(net):
    from paper_1501_06211_gb300 import ddel
    x, _ = batch(1)
    y = torch.zeros((N, COUT, H, W), dtype=torch.float32, device="cuda")
    assert ddel.ddel_cnn_forward(net, torch.as_tensor(x, device="cuda"), N, y) == 0
    ref = cnn.forward(params(net).astype(float), x.astype(float), COUT)
    assert rel(y.cpu().numpy(), ref) < 1e-5


def test_loss_and_gradient_match_oracle(net):
    from paper_1501_06211_gb300 import ddel
    x, t = batch(2)
    n = ddel.ddel_cnn_num_params(net)
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    code, loss = ddel.ddel_cnn_loss_grad(net, torch.as_tensor(x, device="cuda"),
                                          torch.as_tensor(t, device="cuda"), N, g)
    assert code == 0
    loss_ref, g_ref = cnn.loss_and_grad(params(net).astype(float), x.astype(float), t.astype(float))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    gg = g.cpu().numpy().astype(float)
    assert rel(gg, g_ref) < 1e-4
    off = 0
    for (co, ci, k, _) in cnn.layer_shapes(CIN, COUT):  # every layer, weights and bias
        m = co * ci * k * k + co
        assert rel(gg[off:off + m], g_ref[off:off + m]) < 1e-3
        off += m


def test_adam_step_matches_oracle(net):
    from paper_1501_06211_gb300 import ddel
    x, t = batch(3)
    p0 = params(net)
    assert ddel.ddel_cnn_set_params(net, p0, 0) == 0  # resets the moments
    n = p0.size
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    theta, m, v = p0.astype(float), np.zeros(n), np.zeros(n)
    for step in (1, 2):
        assert ddel.ddel_cnn_loss_grad(net, xd, td, N, g)[0] == 0
        gh = g.cpu().numpy().astype(float)
        assert ddel.ddel_cnn_adam_step(net, 1e-3) == 0
        theta, m, v = cnn.adam_step(theta, gh, m, v, step, lr=1e-3)
        assert np.max(np.abs(params(net) - theta)) < 1e-6
    assert ddel.ddel_cnn_set_params(net, p0, 0) == 0


def test_training_reduces_loss_and_is_deterministic(net):
    from paper_1501_06211_gb300 import ddel
    x, _ = batch(4)
    t = np.tanh(x[:, :1].repeat(COUT, axis=1)).astype(np.float32)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    p0 = params(net)
    runs = []
    for _ in range(2):
        assert ddel.ddel_cnn_set_params(net, p0, 0) == 0
        losses = []
        for _ in range(60):
            code, loss = ddel.ddel_cnn_loss_grad(net, xd, td, N)
            assert code == 0
            losses.append(loss)
            assert ddel.ddel_cnn_adam_step(net, 3e-3) == 0
        runs.append((losses, params(net)))
    assert runs[0][0][-1] < 0.5 * runs[0][0][0]
    assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])
    assert ddel.ddel_cnn_set_params(net, p0, 0) == 0


def test_cnn_argument_errors():
    from paper_1501_06211_gb300 import ddel
    assert ddel.ddel_cnn_create(3, 4, 30, 24, 1)[0] == ddel.DDEL_EINVAL  # H not a multiple of 8
    assert ddel.ddel_cnn_create(3, 4, 32, 24, 0)[0] == ddel.DDEL_EINVAL
    code, h = ddel.ddel_cnn_create(3, 4, 32, 24, 1)
    assert code == 0
    x = torch.zeros((2, 3, 32, 24), dtype=torch.float32, device="cuda")
    y = torch.zeros((2, 4, 32, 24), dtype=torch.float32, device="cuda")
    assert ddel.ddel_cnn_forward(h, x, 2, y) == ddel.DDEL_EINVAL  # batch above max_batch
    ddel.ddel_cnn_destroy(h)


# ------------------------------------------------------------------ learner
def features_reference(rho_f, ne, f, u):
    """The learner's input / target as the header defines them."""
    nx, ny = ne
    Hp, Wp = (nx + 1 + 7) // 8 * 8, (ny + 1 + 7) // 8 * 8
    r = rho_f.reshape(nx, ny)
    pad = np.pad(r, 1, constant_values=np.nan)
    win = np.stack([pad[a:a + nx + 1, b:b + ny + 1] for a in (0, 1) for b in (0, 1)])
    rn = np.nanmean(win, axis=0)
    fx, fy = f[0::2].reshape(nx + 1, ny + 1), f[1::2].reshape(nx + 1, ny + 1)
    fm = np.max(np.abs(f))
    ux, uy = u[0::2].reshape(nx + 1, ny + 1), u[1::2].reshape(nx + 1, ny + 1)
    um = np.max(np.abs(u))
    x = np.zeros((3, Hp, Wp))
    t = np.zeros((4, Hp, Wp))
    x[0, :nx + 1, :ny + 1] = rn
    x[1, :nx + 1, :ny + 1] = fx / fm
    x[2, :nx + 1, :ny + 1] = fy / fm
    t[0, :nx + 1, :ny + 1] = rn * ux / um
    t[1, :nx + 1, :ny + 1] = rn * uy / um
    t[2, :nx + 1, :ny + 1] = (1 - rn) * ux / um
    t[3, :nx + 1, :ny + 1] = (1 - rn) * uy / um
    return x, t


def test_learner_features_match_definition():
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(40, 20, 10, seed=2)
    s = ddel.Solver(cfg)
    L = ddel.Learner(s)
    Hp, Wp = L.grid()
    assert (Hp, Wp) == (48, 24)
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.001, 1.0, 40 * 20)
    u = rng.standard_normal(s.n_dof)
    x = torch.zeros((3, Hp, Wp), dtype=torch.float32, device="cuda")
    t = torch.zeros((4, Hp, Wp), dtype=torch.float32, device="cuda")
    assert ddel.ddel_learner_features(L.h, torch.as_tensor(rho, device="cuda"),
                                      torch.as_tensor(u, device="cuda"), x, t) == 0
    xr, tr = features_reference(rho, (40, 20), s.load_vector(), u)
    assert rel(x.cpu().numpy(), xr) < 1e-6 and rel(t.cpu().numpy(), tr) < 1e-6
    L.close()


def run_topopt(cfg, steps, mode=None, **lopts):
    from paper_1501_06211_gb300 import ddel
    s = ddel.Solver(cfg, tol=1e-8, max_it=20000)
    L = ddel.Learner(s, mode=mode, **lopts) if mode is not None else None
    ne = int(np.prod(cfg["ne"]))
    rho = torch.full((ne,), 0.5, dtype=torch.float64, device="cuda")
    ts = s.topopt_state(rho, 0.5, r_min=1.5, move=0.2, learner=L)
    out = []
    for _ in range(steps):
        st = s.topopt_step(ts)
        out.append((st.iters, st.coarse_k, st.x0_used, ts.compliance, st.relres))
    info = L.info() if L else None
    return out, info, rho.cpu().numpy()


def test_topopt_with_history_and_learned_coarse_space():
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(96, 48, 12, seed=3, bc="mbb")
    steps = 10
    plain, _, rho_p = run_topopt(cfg, steps)
    hist, ih, rho_h = run_topopt(cfg, steps, ddel.DDEL_LEARN_HISTORY, k_history=4)
    lrn, il, rho_l = run_topopt(cfg, steps, ddel.DDEL_LEARN_CNN, train_steps=10, replay=8)
    both, ib, rho_b = run_topopt(cfg, steps, ddel.DDEL_LEARN_CNN_HISTORY, k_history=2, train_steps=5)
    for run in (plain, hist, lrn, both):
        assert all(r[4] <= 1e-8 for r in run)
    # the same designs: every solve meets the tolerance, so the OC updates agree
    for run, rho in ((hist, rho_h), (lrn, rho_l), (both, rho_b)):
        ca, cb = np.array([r[3] for r in plain]), np.array([r[3] for r in run])
        assert np.max(np.abs(ca - cb) / ca) < 1e-5
        assert np.max(np.abs(rho_p - rho)) < 1e-4
    # history coarse space from the second step on, learned one from min_samples on
    assert [r[1] for r in hist][1:] == [min(j, 4) for j in range(1, steps)]
    assert all(r[1] >= 2 for r in lrn[2:]) and ih.samples == 4 and il.samples == 8
    assert all(r[1] >= 4 for r in both[2:]) and ib.samples == steps
    assert il.adam_steps == 10 * steps and il.last_loss >= 0 and ib.adam_steps == 5 * steps
    # what the coarse spaces gain over the plain method once they exist: fewer
    # PCG iterations per Picard solve (previous solutions, and the trained
    # network's fields on their own)
    assert sum(r[0] for r in hist[3:]) < sum(r[0] for r in plain[3:])
    assert sum(r[0] for r in lrn[3:]) < sum(r[0] for r in plain[3:])

"""Selection controller: the FP64 CPU reference is pinned by finite differences (no GPU);
the GPU forward / backward / Adam kernels match it (gpu)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1305_1293_gb300.meshgen import SplitMix64


def _data(n, seed=3):
    rng = SplitMix64(seed)
    X = rng.normal(n * mo.N_FEATURES).reshape(n, mo.N_FEATURES)
    t = rng.normal(n)
    return X, t


def test_param_count():
    assert mo.N_PARAMS == 64 * 24 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_backward_matches_central_differences():
    """The hand-derived backward pass against (L(p + h e_i) - L(p - h e_i)) / 2h."""
    p = mo.init_params(1)
    rng = SplitMix64(9)
    p = p + 0.05 * rng.normal(p.size)          # nonzero biases, W4 away from 0
    X, t = _data(37)
    g = mo.grad(p, X, t)
    idx = np.unique(np.concatenate([np.arange(0, mo.N_PARAMS, 97), [mo.N_PARAMS - 1, mo.N_PARAMS - 65]]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mo.loss(p + e, X, t) - mo.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, i


def test_forward_special_cases():
    """All-zero weights give y = b4; a single active path is a product of weights."""
    p = np.zeros(mo.N_PARAMS)
    p[-1] = 0.75
    X, _ = _data(5)
    assert np.allclose(mo.forward(p, X)[0], 0.75)
    q = mo.unpack(np.zeros(mo.N_PARAMS))
    q["W1"][0, 2] = 2.0
    q["W2"][0, 0] = 3.0
    q["W3"][0, 0] = 0.5
    q["W4"][0] = -1.0
    pp = mo.pack(q)
    x = np.zeros((2, mo.N_FEATURES))
    x[0, 2], x[1, 2] = 1.5, -1.0      # second sample blocked by the first ReLU
    y, _ = mo.forward(pp, x)
    assert np.allclose(y, [-(2.0 * 1.5) * 3.0 * 0.5, 0.0])


def _adam_constant_gradient_error(step, t_max=6):
    """Largest deviation of ``step`` (an Adam update with the adam_step signature) from
    the closed form of Kingma & Ba, "Adam: A Method for Stochastic Optimization" (ICLR
    2015), Algorithm 1, under a constant gradient g.  Then m_t = (1 - b1^t) g and
    v_t = (1 - b2^t) g^2, so the bias-corrected moments are exactly g and g^2 at every t
    and each step moves a parameter by lr g / (|g| + eps): after t steps
    p_0 - t lr g / (|g| + eps).  The gradients include ones of the size of eps, where the
    step is visibly not lr sign(g) (that pins where eps enters), and zero."""
    lr, eps = 1e-3, 1e-8
    g = np.array([1.0, -2.5, 1e3, 1e-8, -3e-9, 0.0, 7e-5])
    p0 = np.linspace(-1.0, 1.0, g.size)
    p, m, v = p0.copy(), np.zeros_like(g), np.zeros_like(g)
    worst = 0.0
    for t in range(1, t_max + 1):
        p, m, v = step(p, g, m, v, t, lr)
        exact = p0 - t * lr * g / (np.abs(g) + eps)
        worst = max(worst, float(np.max(np.abs(p - exact))) / lr)
    return worst


def _adam_impulse_error(step, t_max=6, b1=0.9, b2=0.999):
    """Deviation of ``step`` from the closed form of Adam's recurrences for a gradient g at
    step 1 and zero afterwards: m_t = b1^(t-1) (1 - b1) g and v_t = b2^(t-1) (1 - b2) g^2,
    so the step t update is lr m_t / (1 - b1^t) / (sqrt(v_t / (1 - b2^t)) + eps).  Unlike
    the constant gradient this depends on the two decay rates."""
    lr, eps = 1e-3, 1e-8
    g = np.array([1.0, -2.5, 1e-8, 0.0])
    p0 = np.linspace(-1.0, 1.0, g.size)
    p, m, v = p0.copy(), np.zeros_like(g), np.zeros_like(g)
    exact = p0.copy()
    worst = 0.0
    for t in range(1, t_max + 1):
        p, m, v = step(p, g if t == 1 else np.zeros_like(g), m, v, t, lr)
        mt = b1 ** (t - 1) * (1 - b1) * g
        vt = b2 ** (t - 1) * (1 - b2) * g * g
        exact = exact - lr * (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
        worst = max(worst, float(np.max(np.abs(p - exact))) / lr)
    return worst


def test_adam_closed_form_constant_gradient():
    assert _adam_constant_gradient_error(mo.adam_step) <= 1e-12
    assert _adam_impulse_error(mo.adam_step) <= 1e-12
    # first step: lr sign(g) up to eps for |g| >> eps, half of it for |g| = eps
    p1, _, _ = mo.adam_step(np.zeros(3), np.array([2.0, -1e-8, 1e-8]), np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p1, [-0.01, 0.005, -0.005], rtol=1e-7, atol=0)


def test_adam_pin_catches_planted_mistakes():
    """Plausible mistakes in an Adam step, each planted in a copy of the oracle's update,
    all fail one of the two closed-form pins above."""
    def no_bias_correction(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        return p - lr * m / (np.sqrt(v) + eps), m, v

    def betas_swapped(p, g, m, v, t, lr):
        return mo.adam_step(p, g, m, v, t, lr, b1=0.999, b2=0.9)

    def eps_inside_sqrt(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        return p - lr * (m / (1 - b1 ** t)) / np.sqrt(v / (1 - b2 ** t) + eps), m, v

    def corrected_with_t_minus_1(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        tt = max(t - 1, 1)
        return p - lr * (m / (1 - b1 ** tt)) / (np.sqrt(v / (1 - b2 ** tt)) + eps), m, v

    def moment_without_one_minus_beta(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + g
        v = b2 * v + (1 - b2) * g * g
        return p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps), m, v

    for bad in (no_bias_correction, betas_swapped, eps_inside_sqrt, corrected_with_t_minus_1,
                moment_without_one_minus_beta):
        assert max(_adam_constant_gradient_error(bad), _adam_impulse_error(bad)) > 1e-6, bad.__name__


def test_adam_reduces_loss_cpu():
    p = mo.init_params(2)
    X, _ = _data(64, 5)
    t = X[:, 0] * 0.5 - X[:, 3]
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mo.loss(p, X, t)
    for k in range(1, 201):
        p, m, v = mo.adam_step(p, mo.grad(p, X, t), m, v, k, 1e-2)
    assert mo.loss(p, X, t) < 0.2 * l0


# ------------------------------------------------------------------ GPU kernels
@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch
    return torch, pch


@pytest.mark.gpu
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_gpu_forward_backward_match_cpu(gpu, n):
    torch, pch = gpu
    p = (mo.init_params(4) + 0.05 * SplitMix64(11).normal(mo.N_PARAMS)).astype(np.float32)
    X, t = _data(n, 6)
    X, t = X.astype(np.float32), t.astype(np.float32)
    dev = "cuda"
    pd, xd, td = (torch.from_numpy(a).to(dev) for a in (p, X, t))
    y = torch.empty(n, dtype=torch.float32, device=dev)
    g = torch.empty(mo.N_PARAMS, dtype=torch.float32, device=dev)
    l = torch.empty(1, dtype=torch.float32, device=dev)
    pch.mlp_forward(pd, xd, y)
    pch.mlp_backward(pd, xd, td, g, l)
    torch.cuda.synchronize()
    p64, X64, t64 = p.astype(np.float64), X.astype(np.float64), t.astype(np.float64)
    y_ref = mo.forward(p64, X64)[0]
    g_ref = mo.grad(p64, X64, t64)
    assert np.max(np.abs(y.cpu().numpy() - y_ref)) <= 1e-4 * max(1.0, np.abs(y_ref).max())
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - g_ref)) <= 1e-4 * max(1e-3, np.abs(g_ref).max())
    assert abs(l.item() - mo.loss(p64, X64, t64)) <= 1e-4 * max(1.0, mo.loss(p64, X64, t64))
    # deterministic reduction: bit-identical on a second call
    g2 = torch.empty_like(g)
    pch.mlp_backward(pd, xd, td, g2, l)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


@pytest.mark.gpu
def test_gpu_adam_matches_cpu(gpu):
    torch, pch = gpu
    p = mo.init_params(5).astype(np.float32)
    g = SplitMix64(3).normal(mo.N_PARAMS).astype(np.float32)
    m = np.zeros(mo.N_PARAMS, dtype=np.float32)
    v = np.zeros(mo.N_PARAMS, dtype=np.float32)
    pd, gd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    pc, mc, vc = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in (1, 2, 3):
        pch.mlp_adam(pd, gd, md, vd, t, 1e-3)
        pc, mc, vc = mo.adam_step(pc, g.astype(np.float64), mc, vc, t, 1e-3)
    torch.cuda.synchronize()
    assert np.max(np.abs(pd.cpu().numpy() - pc)) < 1e-6


@pytest.mark.gpu
def test_trained_controller_gain_and_exactness(gpu, oracle_lib, tmp_path):
    """What the trained network gains on a held-out jittered torus of the 1M-face torus'
    family (seeds disjoint from training), with the distances unchanged (any selection
    order gives the exact field, Section 4.3, Remark 2): against the paper's method (fixed
    k = 24 * 2^10, one hop per iteration), against fixed k with the same chaining, and
    against the plain control at the (k, hops, block) the autotuner picks for this very
    mesh by timing full solves.  The network needs no per-mesh tuning; it must beat the
    first two and stay within 15% of the third (the measured ratio is printed)."""
    torch, pch = gpu
    from paper_1305_1293_gb300 import meshgen as mg
    if not pch.load_controller():
        pytest.skip("no trained weights (run paper_1305_1293_gb300.controller_train on a GPU)")
    m = mg.torus(600, 200, seed=mg.SEED_BASE + 77)
    srcs = mg.pick_sources(m, 2, mg.SEED_BASE + 78)
    mesh = pch.Mesh(m.vertices, m.faces)
    tuned = pch.autotune(mesh, int(srcs[0]), cache_path=str(tmp_path / "tune.txt"))
    tk = {"k": tuned["k"], "hops": tuned["hops"], "block": tuned["block"]}
    lk = {"control": pch.CONTROL_LEARNED, "hops": tuned["hops"], "block": tuned["block"]}

    def best_ms(s, kw, reps=3):
        pch.solve(mesh, s, **kw)                                        # builds the graph
        runs = [pch.solve(mesh, s, stats=True, **kw) for _ in range(reps)]
        return min(r[1]["ms_total"] for r in runs), runs[-1][0]

    t_plain = t_learned = t_same = t_tuned = 0.0
    for s in srcs:
        s = int(s)
        tp, plain = best_ms(s, {"k": 24576, "hops": 1}, reps=1)          # the paper's method and k
        ts, _ = best_ms(s, {"k": 24576})                                # fixed k, the same chaining
        tt, _ = best_ms(s, tk)                                          # plain at the tuned setting
        tl, learned = best_ms(s, lk)
        t_plain += tp
        t_same += ts
        t_tuned += tt
        t_learned += tl
        assert np.max(np.abs(learned - plain) / np.maximum(plain, 1e-300)) < 1e-9
        near = np.argsort(learned)[1:301].astype(np.int32)
        ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s, targets=near)
        assert np.max(np.abs(learned[near] - ref[near]) / ref[near]) < 1e-9
    mesh.close()
    print(f"torus 600x200: plain k=24576 one hop {t_plain:.1f} ms, plain k=24576 chained {t_same:.1f} ms, "
          f"plain tuned {tk} {t_tuned:.1f} ms, learned {t_learned:.1f} ms; learned / tuned = "
          f"{t_learned / t_tuned:.3f}, gain {t_plain / t_learned:.1f}x over the paper's method")
    assert t_learned < t_plain
    assert t_learned < t_same
    assert t_learned <= 1.15 * t_tuned

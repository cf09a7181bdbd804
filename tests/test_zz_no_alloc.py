"""The allocation-free controller backward pass (pch_mlp_backward_noalloc) gives the
same gradient and loss as pch_mlp_backward, call after call.

It exists for callers that cannot call cudaMalloc (their own allocator owns the device,
or an allocation mid-loop must never stall or fail); its scratch is one fixed device
array shared by every call.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-4     # the tolerance of the controller's GPU tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch
    return torch, pch


def _case(torch, pch, n, seed):
    from paper_1305_1293_gb300.meshgen import SplitMix64
    rng = SplitMix64(seed)
    npar, nf = pch.mlp_num_params(), pch.mlp_num_features()
    p = (0.2 * rng.normal(npar)).astype(np.float32)
    x = rng.normal(n * nf).reshape(n, nf).astype(np.float32)
    t = rng.normal(n).astype(np.float32)
    return tuple(torch.from_numpy(a).cuda() for a in (p, x, t))


def test_noalloc_matches_allocating_backward_twice(env):
    torch, pch = env
    for call, (n, seed) in enumerate(((4096, 11), (777, 12))):   # two calls in a row
        p, x, t = _case(torch, pch, n, seed)
        g_ref = torch.empty(pch.mlp_num_params(), dtype=torch.float32, device="cuda")
        l_ref = torch.empty(1, dtype=torch.float32, device="cuda")
        g = torch.full_like(g_ref, float("nan"))
        l = torch.full_like(l_ref, float("nan"))
        pch.mlp_backward(p, x, t, g_ref, l_ref)
        pch.mlp_backward_noalloc(p, x, t, g, l)
        torch.cuda.synchronize()
        scale = max(1e-3, g_ref.abs().max().item())
        assert torch.isfinite(g).all(), call
        assert (g - g_ref).abs().max().item() <= REL * scale, call
        assert abs(l.item() - l_ref.item()) <= REL * max(1.0, abs(l_ref.item())), call


def test_noalloc_rejects_more_than_the_limit(env):
    torch, pch = env
    p, x, t = _case(torch, pch, 4097, 13)
    g = torch.zeros(pch.mlp_num_params(), dtype=torch.float32, device="cuda")
    l = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(pch.PchError) as e:
        pch.mlp_backward_noalloc(p, x, t, g, l)
    assert e.value.status == pch.PCH_ERR_CAPACITY
    torch.cuda.synchronize()
    assert g.abs().max().item() == 0.0        # nothing computed

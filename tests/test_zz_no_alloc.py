"""boruta_binom_tails_noalloc through the C ABI: the entry point for callers
that may not allocate device memory (their own allocator has reserved the
GPU, or cudaMalloc is not allowed on their path).  It must give exactly the
results of boruta_binom_tails, call after call, while the library keeps its
table in a fixed device array.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _queries(seed):
    rng = np.random.default_rng(seed)
    t = rng.integers(0, 127, size=3000).astype(np.int32)
    t[:4] = [0, 1, 126, 63]
    h = np.array([int(rng.integers(0, tt + 2)) for tt in t], dtype=np.int32)
    return t, h


def test_noalloc_matches_allocating_entry_point_twice():
    import torch

    import __graft_entry__
    from paper_2605_09950_gb300 import boruta

    __graft_entry__.build()
    dev = torch.device("cuda:0")
    for call, seed in enumerate((1, 2)):  # two calls in a row share the fixed array
        t_np, h_np = _queries(seed)
        t = torch.from_numpy(t_np).to(dev)
        h = torch.from_numpy(h_np).to(dev)
        want_a, want_r = boruta.boruta_binom_tails(t, h)
        got_a = torch.full((t.numel(),), -1.0, dtype=torch.float64, device=dev)
        got_r = torch.full_like(got_a, -1.0)
        boruta.boruta_binom_tails_noalloc(t, h, got_a, got_r)
        np.testing.assert_array_equal(got_a.cpu().numpy(), want_a.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(got_r.cpu().numpy(), want_r.cpu().numpy(), err_msg=f"call {call}")


def test_noalloc_rejects_t_beyond_table():
    import torch

    from paper_2605_09950_gb300 import boruta

    dev = torch.device("cuda:0")
    t = torch.tensor([5, 127], dtype=torch.int32, device=dev)
    h = torch.tensor([2, 3], dtype=torch.int32, device=dev)
    a = torch.empty(2, dtype=torch.float64, device=dev)
    r = torch.empty_like(a)
    with pytest.raises(boruta.BorutaError, match="126"):
        boruta.boruta_binom_tails_noalloc(t, h, a, r)
    # a good call right after a rejected one still works (error word is cleared)
    t2 = torch.tensor([5], dtype=torch.int32, device=dev)
    h2 = torch.tensor([2], dtype=torch.int32, device=dev)
    a2 = torch.empty(1, dtype=torch.float64, device=dev)
    r2 = torch.empty_like(a2)
    boruta.boruta_binom_tails_noalloc(t2, h2, a2, r2)
    wa, wr = boruta.boruta_binom_tails(t2, h2)
    assert a2.item() == wa.item() and r2.item() == wr.item()


def test_noalloc_calls_leave_free_memory_unchanged():
    """After a first call on the device (which loads the module holding the
    fixed array), further calls -- good ones and a rejected one -- allocate
    no device memory: the device's free memory is the same before and
    after.  Every tensor the calls use is allocated before the first
    reading."""
    import torch

    from paper_2605_09950_gb300 import boruta

    dev = torch.device("cuda:0")
    t_np, h_np = _queries(3)
    t = torch.from_numpy(t_np).to(dev)
    h = torch.from_numpy(h_np).to(dev)
    a = torch.empty(t.numel(), dtype=torch.float64, device=dev)
    r = torch.empty_like(a)
    tb = torch.tensor([127], dtype=torch.int32, device=dev)
    hb = torch.tensor([0], dtype=torch.int32, device=dev)
    ab = torch.empty(1, dtype=torch.float64, device=dev)
    rb = torch.empty_like(ab)
    boruta.boruta_binom_tails_noalloc(t, h, a, r)  # warm-up: first use on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(3):
        boruta.boruta_binom_tails_noalloc(t, h, a, r)
        with pytest.raises(boruta.BorutaError, match="126"):
            boruta.boruta_binom_tails_noalloc(tb, hb, ab, rb)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0

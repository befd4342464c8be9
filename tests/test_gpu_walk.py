"""GPU parity of the parallel random walk (Section 5.4) through the C ABI.

Positions are integers and every decision is exact on both sides (integer
likelihoods, SplitMix64 numbers), so positions after each step and the
number of cell evaluations must equal the oracle's bit for bit."""
import numpy as np
import pytest

import meshgen as mg
from oracle import walk as W

pytestmark = pytest.mark.gpu


def _run_gpu(act, keys, steps, seed, variant, batch=576, threads=0, first_step=0):
    import torch
    import paper_1805_08893_gb300 as gp
    a = torch.from_numpy(act.view(np.int32)).cuda()
    pos = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    scratch = torch.empty_like(pos)
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    gp.gp_random_walk(a, pos, scratch, cnt, steps, seed, variant, first_step=first_step, batch_agents=batch,
                      threads=threads)
    torch.cuda.synchronize()
    return pos.cpu().numpy().view(np.uint32), cnt.cpu().numpy()


@pytest.mark.parametrize("variant,batch,threads", [("naive", 256, 0), ("warp", 576, 0), ("sort", 576, 256),
                                                    ("hash", 576, 256), ("phash", 576, 128), ("hash", 1024, 512),
                                                    ("sort", 64, 64), ("hash", 96, 32)])
def test_small_grid_steps_match_oracle(variant, batch, threads):
    act = mg.walk_activity(5, 48, 40)
    keys = mg.walk_agents(5, 6000, 48, 40)  # ~3 agents per cell: plenty of reuse in a batch
    want_pos, hist = W.run(act, keys, 3, 1234)
    got, cnt = _run_gpu(act, keys, 3, 1234, variant, batch, threads)
    assert np.array_equal(got, want_pos)
    evals = sum(int(W.batch_invocations(h, variant, batch).sum()) for h in hist[:3])
    assert int(cnt[0]) == evals
    assert int(cnt[2]) == 0


def test_steps_can_be_split_across_calls():
    act = mg.walk_activity(6, 33, 29)
    keys = mg.walk_agents(6, 2000, 33, 29)
    want, _ = W.run(act, keys, 4, 77)
    mid, _ = _run_gpu(act, keys, 3, 77, "hash")
    got, _ = _run_gpu(act, mid, 1, 77, "hash", first_step=3)
    assert np.array_equal(got, want)


def test_full_size_sampled():
    # the paper's configuration: 256 x 256 grid, 300,000 agents; one step, sampled agents
    act = mg.walk_activity(1)
    keys = mg.walk_agents(1)
    got, cnt = _run_gpu(act, keys, 1, 42, "hash", 576, 256)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(keys), size=300, replace=False).tolist():
        k = int(keys[i])
        dx, dy = W.choose(W.cell_moves(act, k >> 16, k & 0xFFFF), W.splitmix64(42 ^ i))
        want = (((k >> 16) + dx) % 256) << 16 | (((k & 0xFFFF) + dy) % 256)
        assert int(got[i]) == want, i
    assert int(cnt[0]) == int(W.batch_invocations(keys, "hash", 576).sum())


def test_zero_field_stays_and_bad_arguments_fail():
    import paper_1805_08893_gb300 as gp
    act = np.zeros((20, 20), dtype=np.uint32)
    keys = mg.walk_agents(2, 300, 20, 20)
    got, _ = _run_gpu(act, keys, 2, 5, "warp", 96)
    assert np.array_equal(got, keys)
    with pytest.raises(gp.GpError):
        _run_gpu(np.zeros((10, 10), dtype=np.uint32), keys, 1, 5, "hash")  # grid smaller than 17
    with pytest.raises(gp.GpError):
        _run_gpu(act, keys, 1, 5, "hash", batch=100)  # not a multiple of 32

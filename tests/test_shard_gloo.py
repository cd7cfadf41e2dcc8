"""N>1 host logic on CPU with the gloo backend, world size 2: time-step partitioning, the
max-over-ranks step time, and the adjoint's one exchange step (the gradient all-reduce). Each rank
computes its slice's gradient with the oracle and the all-reduced sum must equal the gradient of the
whole observation."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2005_09316_b300 import shard  # noqa: E402


@pytest.mark.parametrize("n_time,world", [(14, 1), (14, 2), (14, 3), (5, 8), (0, 2), (1, 4)])
def test_time_partition_covers_every_step_once(n_time, world):
    seen = []
    for r in range(world):
        t0, t1 = shard.time_partition(n_time, world, r)
        assert 0 <= t0 <= t1 <= n_time
        seen.extend(range(t0, t1))
    assert seen == list(range(n_time))
    sizes = [np.subtract(*shard.time_partition(n_time, world, r)[::-1]) for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _problem():
    import synth
    obs = synth.make_obs(41, 8, 3, synth.uniform_channels(167e6, 80e3, 6), layout="mwa")
    sky = synth.make_sky(42, 3, 2, 1, fov=10 * synth.DEG, shape_nmax=4)
    gains = synth.make_gains(43, obs.n_ant).astype(np.complex128)
    rng = np.random.default_rng(44)
    data = rng.normal(size=(obs.n_time, obs.n_base, obs.n_chan)) + 1j * rng.normal(size=(obs.n_time, obs.n_base, obs.n_chan))
    return obs, sky, gains, data


def _slice_grad(obs, sky, gains, data, t0, t1):
    import oracle
    rows = np.arange(t0 * obs.n_base, t1 * obs.n_base)
    uvw = obs.uvw.reshape(-1, 3)[rows]
    rt, rb = rows // obs.n_base, rows % obs.n_base
    V = oracle.predict(uvw, obs.freq, obs.dec0, sky)
    G = oracle.gain_product(rt, rb, obs.ant1, obs.ant2, gains, obs.n_chan)
    D = data.reshape(-1, obs.n_chan)[rows]
    R = D - G * V
    gr = oracle.grad(uvw, obs.freq, obs.dec0, sky, np.conj(G) * R)
    gr["loss"] = np.array([np.sum(np.abs(R) ** 2)])
    return gr


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        obs, sky, gains, data = _problem()
        t0, t1 = shard.time_partition(obs.n_time, world, rank)
        local = {k: torch.as_tensor(np.atleast_1d(v).astype(np.float64)) for k, v in
                 _slice_grad(obs, sky, gains, data, t0, t1).items()}
        summed = shard.allreduce_grads(local)
        ms = shard.max_over_ranks(10.0 + rank)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), ms=ms, **{k: v.numpy() for k, v in summed.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_two_ranks_gradient_allreduce_and_max_time(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    obs, sky, gains, data = _problem()
    full = _slice_grad(obs, sky, gains, data, 0, obs.n_time)
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert float(got["ms"]) == 10.0 + world - 1
        for k, v in full.items():
            v = np.atleast_1d(v)
            if v.size:
                np.testing.assert_allclose(got[k], v, rtol=1e-10, atol=1e-12 * max(1.0, np.abs(v).max()), err_msg=k)

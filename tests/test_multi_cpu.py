"""World-size-2 gloo test of the multi-beam host logic on CPU: ranks search
disjoint beams (here with the CPU oracle standing in for the device search),
reduce their timings with a max, and the merged candidate list equals the
serial search of every beam."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NBEAMS = 3


def _beam_cands(beam):
    import oracle
    from paper_2110_12749_gb300 import gsp, shard, synth
    nchan, n_in, ts = 64, 6144, 1e-4
    dms = np.arange(0.0, 24.0, 1.0)
    dl, _ = oracle.delays(nchan, 1200.0, 1500.0, ts, dms)
    n_out = n_in - oracle.max_delay(dl)
    p = synth.Pulse(dm=9.0, t0=1000 + 700 * beam, width=3, snr=20.0,
                    amp=synth.pulse_amplitude(20.0, 16.0, nchan, 3), delays=dl[9])
    x = synth.filterbank(nchan, n_in, synth.beam_seed(beam), 128.0, 16.0, pulses=[p],
                         beam=beam, threads=1)
    D = oracle.dedisperse(x, n_in, dl)
    c, _ = oracle.search_rows(D, block_len=1024, window_len=1024)
    out = np.zeros(len(c), dtype=gsp.CAND_DTYPE)
    for f in ("dm_idx", "width", "t", "snr"):
        out[f] = c[f]
    return shard.label_beam(out, beam)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2110_12749_gb300 import gsp, shard
    mine = [_beam_cands(b) for b in shard.beams_for_rank(NBEAMS, rank, world)]
    local = shard.merge_candidates(mine, gsp.CAND_DTYPE)
    tmax = shard.max_over_ranks(1.0 + rank, dist)
    merged = shard.gather_candidates(local, dist, gsp.CAND_DTYPE)
    if rank == 0:
        q.put((tmax, merged))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_beam_sharding():
    from paper_2110_12749_gb300 import gsp, shard
    assert shard.beams_for_rank(5, 0, 2) == [0, 2, 4]
    assert shard.beams_for_rank(5, 1, 2) == [1, 3]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tmax, merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0
    serial = shard.merge_candidates([_beam_cands(b) for b in range(NBEAMS)], gsp.CAND_DTYPE)
    assert len(merged) == len(serial) > 0
    assert (merged == serial).all()
    assert sorted(set(merged["beam"].tolist())) == list(range(NBEAMS))

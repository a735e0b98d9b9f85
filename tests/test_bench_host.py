"""Host logic of bench.py without a GPU: the max-over-ranks / sum-over-ranks
aggregation of independent replicas (two gloo ranks on CPU) and the parsing
of sampled nvidia-smi clock lines."""
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t, v = bench.reduce_max_sum(1.5 + rank, 1000 * (rank + 1), ws)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_reduce_max_sum_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, v in out:
        assert t == 2.5 and v == 3000.0


def test_reduce_single_rank_is_identity():
    assert bench.reduce_max_sum(3.0, 7, 1) == (3.0, 7)


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_sampler_parses_reasons():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("0, 1900, 2032, 700.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                       "0, 1800, 2032, 1099.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                       "0, 2000, 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = s.stop()
    assert c["sm_mhz"] == 1900 and c["sm_max_mhz"] == 2032 and c["reasons"] == ["sw_power_cap"]


def test_stored_traffic_tracks_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from the committed capture only while
    the image pass's source is the one that was captured."""
    b = bench
    h = b.image_pass_source_hash()
    assert len(h) == 64 and h == b.image_pass_source_hash()
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "k_image_hess_lung_ct.md"
    prof.write_text(f"x\ntraffic_bytes_per_launch: 123\nimage_pass_source_sha256: {h}\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "image_pass_source_hash", lambda: h)
    assert b.stored_traffic("lung_ct") == 123.0
    assert b.stored_traffic("thorax_abd") is None  # no capture of that workload here
    prof.write_text("x\ntraffic_bytes_per_launch: 123\nimage_pass_source_sha256: 00\n")
    assert b.stored_traffic("lung_ct") is None


def test_shard_pairs_partitions_and_balances():
    sizes = [((k * 37) % 129 + 64) ** 3 for k in range(64)]
    for ws in (1, 2, 3, 8):
        shards = [bench.shard_pairs(sizes, ws, r) for r in range(ws)]
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(64))  # every pair exactly once
        loads = [sum(sizes[i] for i in sh) for sh in shards]
        assert max(loads) - min(loads) <= max(sizes)  # greedy bound

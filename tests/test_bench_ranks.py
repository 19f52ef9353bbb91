"""bench.py's host-side arithmetic on CPU.  Multi-rank (gloo, world size 2): timings are
the slowest rank's, and N replicas of one circuit each make N circuits per that time (the
GPU path differs only in the tensors' device, NCCL).  The algorithmic flop count behind
the FP32 roofline, recounted from the oracle's own gate list."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        # rank r took (1 + r) ms on the device and (5 - r) s of wall time
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank], dist, 'cpu')
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: [2.0, 5.0], 1: [2.0, 5.0]}


def test_single_process_and_replica_value():
    assert bench.max_over_ranks([0.5, 7], None, 'cpu') == [0.5, 7.0]
    assert bench.whole_job_s_per_circuit(0.66, 1) == 0.66
    assert bench.whole_job_s_per_circuit(0.66, 4) == pytest.approx(0.165)


def test_algorithmic_flops_of_the_34q_circuit():
    """2 real operations per amplitude for each square root of X or Y (an unscaled
    rotation; its scalar is applied once per circuit), 2 for each T (half the amplitudes
    times (1 + i)/sqrt2), none for CZ; the H layer is the generated uniform state: 464 per
    amplitude for the 34-qubit depth-30 circuit."""
    from oracle import circuit as oc
    from paper_1804_04797_gb300 import inputs, sv
    lat = inputs.C34
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    kinds = [k for (k, _a, _b, layer) in gates if layer > 0]
    want = 2 * sum(k in ('SX', 'SY') for k in kinds) + 2 * sum(k == 'T' for k in kinds)
    assert 'H' not in kinds and want == 464
    assert bench.algorithmic_flops_per_amplitude(sv.sv_generate_circuit(lat)) == want

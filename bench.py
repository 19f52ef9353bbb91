"""Benchmark: seconds per circuit for the 34-qubit depth-30 lattice circuit on one GB300.

One step = one full simulation of the 6x6-minus-two-corners lattice circuit (478 gates
including the layer-0 H layer) from |0...0> on a 128 GiB complex64 state: plan upload,
every tile pass, nothing skipped.  The state (137 GB) is far larger than L2 (129 MB), so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default run prints ONE JSON line: the headline (plain path), the tensor-core paths
beside it (with and without their norm restore), the per-pass times, the roofline of the
dominant kernel, an accuracy block at 30 qubits against the complex128 oracle (rel-L2,
1 - fidelity and norm error of every path), the oracle's own times (16 and 30 qubits
measured, single-thread and all cores; 34 qubits extrapolated, stated as such) and the
secondary workloads (uneven batch, 42-qubit cut-branch amplitudes, 34-qubit amplitudes by
the inner product, 28-qubit full state by the tensor form), each with its own config.

For N > 1 (torchrun, one rank per GPU) every rank simulates its own replica of the
circuit (the state-vector simulation does not shard: one 34-qubit state fills one GPU)
and value = N circuits / the slowest rank's time.
--impl reference times the CPU oracle (the only reference this method has) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = '34q depth-30 s/circuit & %HBM roofline; fused-TC vs plain at rel-L2≤1e-5'
UNIT = 's/circuit'


def max_over_ranks(values, dist, device):
    """Each value's maximum over the ranks (every rank gets the same list): timings are
    the slowest rank's.  dist None: a single process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_s_per_circuit(slowest_s_per_circuit, world):
    """N replicas each simulate one circuit per step and the step ends with the slowest:
    N circuits per slowest time, i.e. the slowest time / N seconds per circuit."""
    return slowest_s_per_circuit / world


def _peaks():
    """(HBM GB/s, bf16 dense TFLOP/s burst, kind) from MEASURED_PEAKS.json, else the
    fallback figures."""
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            p = json.load(f)
        return float(p['hbm_gbs']), float(p['bf16_tflops']), 'measured'
    except Exception:
        return 6800.0, 1900.0, 'fallback'


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic byte of the
# dominant kernels, from one ncu capture each on one pass of the 28-qubit depth-30 circuit
# (2^28 amplitudes); a pass moves each amplitude once in and once out, so traffic scales
# with the amplitudes.
TRAFFIC_PER_ALGORITHMIC_BYTE = {
    'sv_pass (pipelined)': (2.147896576e9 + 2.086447616e9) / (16.0 * 2 ** 28),
    'sv_pass': (2.147776e9 + 2.128476e9) / (16.0 * 2 ** 28),
    'fused_pass_kernel<f16>': (2.147810e9 + 2.087095e9) / (16.0 * 2 ** 28),
}
SMS, FP32_LANES_PER_SM = 152, 128
# nominal dense tensor rates relative to bf16 (2.25 PFLOP/s): fp16 the same, tf32 1.1
TENSOR_RATIO = {'f16x3': 1.0, 'tf32x3': 1.1 / 2.25}


def algorithmic_flops_per_amplitude(gates):
    """Real additions and multiplications the gate list needs per amplitude: a square root
    of X or Y is a scalar e^{+-i pi/4} 2^{-1/2} (applied once per circuit) times an
    unscaled rotation that updates a pair with 4 real additions (2 per amplitude), H a
    pair with 4 additions and 4 multiplications by 1/sqrt2 (4 per amplitude), T and its
    adjoint multiply half the amplitudes by (1 +- i)/sqrt2 (2 additions + 2
    multiplications each: 2 per amplitude); Z, CZ and the projectors change signs or zero
    and take none.  The leading layer of H on a fresh state is the generated uniform
    state."""
    kinds = [int(k) for k in gates['kind']]
    i = 0
    seen = set()
    while i < len(kinds) and kinds[i] == 0 and int(gates['q0'][i]) not in seen:
        seen.add(int(gates['q0'][i]))
        i += 1
    rest = kinds[i:]
    return 2.0 * sum(k in (2, 3, 9, 10) for k in rest) + 4.0 * sum(k == 0 for k in rest) + \
        2.0 * sum(k in (1, 8) for k in rest)


class Clocks:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.gpu), '--query-gpu=' + self.FIELDS,
                 '--format=csv,noheader,nounits', '-lms', '200'],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for l in getattr(self, 'lines', []):
            f = [x.strip() for x in l.split(',')]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == 'active':
                    reasons.add(name)
        if not sm:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': [], 'samples': 0}
        return {'sm_mhz': statistics.median(sm), 'sm_max_mhz': max(mx), 'reasons': sorted(reasons),
                'samples': len(sm)}


# ---- the oracle's times (CPU, complex128) --------------------------------------------

def _lat_args(lat):
    return lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed


def _oracle_sample():
    """Time the CPU oracle on a bounded sample: the 26-qubit lattice circuit of the same
    construction (6x5 minus its four corners) at depth 30, extrapolated to the 34-qubit
    circuit by gate count x state size (the oracle's cost is one full sweep per gate; the
    34-qubit state itself would need 256 GiB of host memory)."""
    from oracle import circuit as oc
    from oracle import csim
    from paper_1804_04797_gb300 import inputs
    csim.build()
    lat = inputs.lattice_for(6, 5, 30, seed=0, removed=[(0, 0), (0, 4), (5, 0), (5, 4)])
    n, gates = oc.generate(*_lat_args(lat))
    n_full, gates_full = oc.generate(*_lat_args(inputs.C34))
    t0 = time.perf_counter()
    csim.run(n, gates)
    dt = time.perf_counter() - t0
    scale = (len(gates_full) * 2.0 ** n_full) / (len(gates) * 2.0 ** n)
    return dt * scale, dt, csim.threads(), scale, (
        'EXTRAPOLATED: oracle (complex128 C, OpenMP, %d threads) on the 26-qubit depth-30 circuit (%d gates, '
        '%.2f s measured), scaled by gates x 2^n (factor %.1f) to 478 gates x 2^34' % (csim.threads(), len(gates),
                                                                                         dt, scale))


def oracle_times():
    """The oracle measured directly: the 16-qubit circuit single-thread and on all host
    cores, the 30-qubit circuit on all cores (its state is returned for the accuracy
    block), a single-thread sample of the 30-qubit circuit (its first gates, extrapolated
    by gate count, stated as such), and the 34-qubit figure extrapolated from the
    30-qubit all-core time."""
    from oracle import circuit as oc
    from oracle import csim
    from paper_1804_04797_gb300 import inputs
    csim.build()
    cores = csim.threads()
    out = {'cores': cores, 'nproc': os.cpu_count()}
    n16, g16 = oc.generate(*_lat_args(inputs.C16))
    out['16q_d10'] = {'gates': len(g16)}
    for label, th in (('all_cores', cores), ('single_thread', 1)):
        csim.set_threads(th)
        t0 = time.perf_counter()
        for _ in range(20):
            csim.run(n16, g16)
        out['16q_d10']['s_per_circuit_' + label] = (time.perf_counter() - t0) / 20
    csim.set_threads(cores)
    n30, g30 = oc.generate(*_lat_args(inputs.C30))
    t0 = time.perf_counter()
    want = csim.run(n30, g30)
    out['30q_d20'] = {'s_per_circuit_all_cores': time.perf_counter() - t0, 'gates': len(g30),
                      'measured': 'whole circuit'}
    # single thread: the first gates only (a full single-thread run takes tens of minutes)
    k = 4
    csim.set_threads(1)
    t0 = time.perf_counter()
    csim.run(n30, g30[:k])
    dt = time.perf_counter() - t0
    csim.set_threads(cores)
    out['30q_d20']['single_thread_sample'] = {
        'gates_timed': k, 's_measured': dt, 's_per_circuit_extrapolated': dt * len(g30) / k,
        'note': 'EXTRAPOLATED by gate count from the first %d of %d gates' % (k, len(g30))}
    n34, g34 = oc.generate(*_lat_args(inputs.C34))
    scale = (len(g34) * 2.0 ** n34) / (len(g30) * 2.0 ** n30)
    out['34q_d30'] = {'s_per_circuit_all_cores': out['30q_d20']['s_per_circuit_all_cores'] * scale,
                      'extrapolated': True, 'scale_factor': scale,
                      'note': 'EXTRAPOLATED from the measured 30-qubit all-core time by gates x 2^n '
                              '(the 34-qubit complex128 state needs 256 GiB of host memory)'}
    return out, want


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    times = []
    for _ in range(args.warmup):
        _oracle_sample()
    desc, cores, scale = '', 0, 0.0
    for _ in range(args.steps):
        v, _dt, cores, scale, desc = _oracle_sample()
        times.append(v)
    value = statistics.median(times)
    line = {
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': value * 1e3, 'higher_is_better': False,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'c128', 'data': 'synthetic',
        'config': {'workload': '34-qubit 6x6-minus-corners lattice circuit, depth 30, seed 0 (478 gates)',
                   'sample': 'bounded CPU sample, extrapolated'},
        'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': cores, 'kind': 'oracle', 'sample': desc,
                         'extrapolated': True, 'scale_factor': scale},
        'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---- secondary workloads ----------------------------------------------------------------

def batch_workload(steps, warmup, variants=('default',)):
    """The uneven batch (512 circuits, 16..24 qubits, depth 10..24): circuits/s of the
    graph-captured batch against one-at-a-time launches of the same kernels.  Variants:
    'default' (24-qubit circuits on plan kernels, the rest in the persistent launch),
    'jit' (every circuit on kernels compiled for its plan; the first call compiles ~3000
    pass kernels), 'interp' (the interpreting kernel only), 'small' (512 circuits of 12..16
    qubits, where one-at-a-time launches are bound by launch latency).  Timed without the
    per-circuit statistics on both sides (one extra call checks the norms)."""
    import numpy as np
    import torch
    from paper_1804_04797_gb300 import inputs, sv

    def graph(lats, jit):
        opts = sv.options(autotune=1, jit=jit)
        for _ in range(max(1, warmup)):
            sv.sv_apply_batch(lats, opts, stats=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            sv.sv_apply_batch(lats, opts, stats=False)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        stats = sv.sv_apply_batch(lats, opts)
        tile_bits, on_plan_kernels, persistent = sv.sv_batch_config()
        sv.sv_batch_free()
        tuned = {'tile_bits': tile_bits, 'circuits_on_plan_kernels': on_plan_kernels,
                 'circuits_in_persistent_launch': persistent}
        return dt, float(np.max(np.abs(stats[:, 0] - 1.0))), tuned

    def sequential(lats, jit):
        hs = [sv.sv_create(l.n_qubits, sv.options(jit=jit)) for l in lats]
        gl = [sv.sv_generate_circuit(l) for l in lats]
        for h, g in zip(hs, gl):
            sv.sv_reset(h)
            sv.sv_apply_circuit(h, g)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h, g in zip(hs, gl):
            sv.sv_reset(h)
            sv.sv_apply_circuit(h, g)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for h in hs:
            sv.sv_destroy(h)
        return dt

    def compare(lats, jit):
        g, err, tuned = graph(lats, jit)
        q = sequential(lats, jit)
        return {'graph_s_per_batch': g, 'circuits_per_s': len(lats) / g, 'sequential_s_per_batch': q,
                'speedup_vs_sequential': q / g, 'max_norm_err': err, 'tuned_configuration': tuned}

    lats = inputs.batch(512)
    out = {'metric': 'uneven batch circuits/s (graph-captured batch vs one-at-a-time)', 'unit': 'circuits/s',
           'config': {'workload': '512 circuits, 16..24 qubits, depth 10..24, seed 180404797',
                      'state_bytes': 8 * sum(2 ** l.n_qubits for l in lats), 'autotune': 1}}
    jits = {'default': 0, 'jit': 1, 'interp': -1}
    for v in variants:
        if v == 'small':
            out['small'] = {'workload': '512 circuits, 12..16 qubits, depth 10..24, default options',
                            **compare(inputs.batch(512, n_min=12, n_max=16), 0)}
        else:
            out[v] = compare(lats, jits[v])
    out['value'] = out[variants[0]]['circuits_per_s']
    return out


def branch_workload(steps, warmup, paths=('plain', 'tf32x3', 'plain_full_decomposition')):
    """The amplitude task: 64 amplitudes of the 42-qubit 6x7 depth-10 circuit by the cut
    decomposition (t = 10 crossing CZs).  Default: the last layer's 3 crossings are output
    signs and 2 are implicit, so the halves are 21 + 7 and 21 + 5 qubits and 2^5 terms are
    summed per amplitude; full_decomposition: two 31-qubit batched half-states, 2^10
    terms."""
    import torch
    from paper_1804_04797_gb300 import inputs, sv
    lat = inputs.C42
    bits = inputs.bitstrings(lat.n_qubits, 64, seed=2)
    out = {}
    spec = {'plain': (sv.SV_PREC_PLAIN, False), 'tf32x3': (sv.SV_PREC_TF32X3, False),
            'plain_full_decomposition': (sv.SV_PREC_PLAIN, True)}
    for name in paths:
        prec, full = spec[name]
        o = sv.options(precision=prec)
        for _ in range(max(1, warmup)):
            sv.sv_branch_amplitudes(lat, inputs.C42_HALF_A, bits, o, full_decomposition=full)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            amps = sv.sv_branch_amplitudes(lat, inputs.C42_HALF_A, bits, o, full_decomposition=full)
        out[name] = {'s_per_task': (time.perf_counter() - t0) / steps, 'amp0': [amps[0].real, amps[0].imag],
                     'counts': sv.sv_branch_counts(lat, inputs.C42_HALF_A, full)}
    return {'metric': '42q cut-branch amplitude task, s per 64 amplitudes', 'unit': 's/task',
            'value': min(v['s_per_task'] for v in out.values()),
            'config': {'workload': '6x7 lattice, depth 10, cut rows 2|3, t = 10, 64 bitstrings (seed 2)'},
            'paths': out}


def tensor_workload(steps, warmup):
    """The full 28-qubit state (4x7 lattice, depth 10) from the cut decomposition in tensor
    form: two batched half-states (14 + t qubits) and the branch sum of their outer
    products, a complex (2^14 x 2^t) x (2^t x 2^14) product written as 2^28 amplitudes --
    on the CUDA cores (plain) and on the tensor cores (TF32x3 tcgen05 GEMM), for the
    default decomposition and the full one (every crossing CZ summed: 2^7 branches)."""
    import numpy as np
    import torch
    from paper_1804_04797_gb300 import inputs, sv
    lat = inputs.C28
    n = lat.n_qubits
    hbm_peak, bf16_peak, _ = _peaks()
    out = {}
    h = sv.sv_create(n)
    try:
        for full in (False, True):
            counts = sv.sv_branch_counts(lat, inputs.C28_HALF_A, full_decomposition=full)
            tf = counts[4]
            for name, opts in (('cuda_cores', None), ('tensor_cores', sv.options(precision=sv.SV_PREC_TF32X3))):
                for _ in range(max(1, warmup)):
                    sv.sv_branch_full_state(lat, inputs.C28_HALF_A, h, opts, full_decomposition=full)
                torch.cuda.synchronize()
                sv.sv_set_profiling(h, True)
                t0 = time.perf_counter()
                for _ in range(steps):
                    sv.sv_branch_full_state(lat, inputs.C28_HALF_A, h, opts, full_decomposition=full)
                torch.cuda.synchronize()
                dt = (time.perf_counter() - t0) / steps
                ms, _ = sv.sv_get_launch_times(h)
                sv.sv_set_profiling(h, False)
                norm2, _ = sv.sv_norm(h)
                prod_ms = float(np.mean(ms)) if len(ms) else float('nan')
                r = {'s_per_state': dt, 'product_ms': prod_ms, 'norm_err': norm2 - 1.0, 'summed_branch_bits': tf,
                     'product_hbm_gbs': 8.0 * 2 ** n / (prod_ms * 1e-3) / 1e9,
                     'product_hbm_frac': 8.0 * 2 ** n / (prod_ms * 1e-3) / 1e9 / hbm_peak}
                if name == 'tensor_cores':
                    kpad = max(32, -(-2 * 2 ** tf // 32) * 32)
                    na = nb = n // 2
                    tflops = 3 * 2 * 2 ** nb * 2 * 2 ** na * kpad / (prod_ms * 1e-3) / 1e12
                    r['tensor'] = {'achieved': tflops, 'unit': 'TFLOP/s', 'peak': bf16_peak * TENSOR_RATIO['tf32x3'],
                                   'frac': tflops / (bf16_peak * TENSOR_RATIO['tf32x3']),
                                   'note': 'executed TF32x3 products (3 x 2 M N K, K padded to %d)' % kpad}
                out[('full_' if full else '') + name] = r
    finally:
        sv.sv_destroy(h)
    best = out['cuda_cores']['s_per_state']
    return {'metric': '28q full state by the tensor form of the cut decomposition, s per state',
            'value': best, 'unit': 's/state', 'paths': out,
            'config': {'workload': '4x7 lattice, depth 10, cut rows 1|2 (default decomposition: 2^4 summed '
                                   'branches; full: 2^7)',
                       'counts': sv.sv_branch_counts(lat, inputs.C28_HALF_A)}}


def inner_workload(steps, warmup):
    """Task 2 by the inner product: amplitudes of the 34-qubit depth-30 circuit cut after
    layer 15, <U2^dagger x | U1 H^n 0> for 4 bitstrings (one forward state, one backward
    state per bitstring; two 128 GiB states).  s per amplitude, whole call timed."""
    import numpy as np
    import torch
    from paper_1804_04797_gb300 import inputs, sv
    lat = inputs.C34
    bits = np.array(inputs.bitstrings(lat.n_qubits, 4, seed=2), dtype=np.uint64)
    for _ in range(max(1, warmup)):
        sv.sv_amplitudes_by_inner_product(lat, 15, bits)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        amps = sv.sv_amplitudes_by_inner_product(lat, 15, bits)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {'metric': '34q depth-30 amplitude by forward/backward inner product, s per amplitude',
            'value': dt / len(bits), 'unit': 's/amplitude', 's_per_call': dt,
            'amp0': [float(amps[0].real), float(amps[0].imag)],
            'config': {'workload': '6x6-minus-corners lattice, depth 30, cut after layer 15, 4 bitstrings (seed 2)'}}


def accuracy_30q(want, stream):
    """Every path on the 30-qubit depth-20 circuit against the complex128 oracle state:
    rel-L2, 1 - fidelity, norm error (fp64 reduction), and the path's time (one warm run,
    then one timed)."""
    import numpy as np
    import torch
    from paper_1804_04797_gb300 import inputs, sv
    lat = inputs.C30
    n = lat.n_qubits
    g = sv.sv_generate_circuit(lat)
    modes = [('plain', dict()), ('tf32x3', dict(precision=sv.SV_PREC_TF32X3)),
             ('f16x3', dict(precision=sv.SV_PREC_F16X3)),
             ('tf32x3_raw', dict(precision=sv.SV_PREC_TF32X3, norm_restore=-1)),
             ('f16x3_raw', dict(precision=sv.SV_PREC_F16X3, norm_restore=-1))]
    out = {}
    want_norm2 = float(np.vdot(want, want).real)
    chunk = 1 << 26
    for name, kw in modes:
        h = sv.sv_create(n, sv.options(stream=stream.cuda_stream, **kw))
        try:
            sv.sv_apply_circuit(h, g)
            torch.cuda.synchronize()
            sv.sv_reset(h)
            t0 = time.perf_counter()
            sv.sv_apply_circuit(h, g)
            norm2, sp2 = sv.sv_norm(h)
            dt = time.perf_counter() - t0
            psi = sv.sv_copy_state(h, n)
        finally:
            sv.sv_destroy(h)
        d2, dot, p2 = 0.0, 0j, 0.0
        for i in range(0, 1 << n, chunk):
            a = psi[i:i + chunk].astype(np.complex128)
            b = want[i:i + chunk]
            d2 += float(np.sum(np.abs(a - b) ** 2))
            dot += complex(np.vdot(b, a))
            p2 += float(np.vdot(a, a).real)
        del psi
        out[name] = {'rel_l2': (d2 / want_norm2) ** 0.5,
                     'one_minus_fidelity': 1.0 - abs(dot) ** 2 / (want_norm2 * p2),
                     'norm_err': norm2 - 1.0, 'n_sum_p2': (2.0 ** n) * sp2, 's_per_circuit': dt}
    return {'workload': '30-qubit 5x6 lattice circuit, depth 20, seed 0 (293 gates), whole state against the '
                        'complex128 oracle', 'paths': out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--qubits', type=int, default=34, help='34 (headline); 30, 28 or 16 for smaller cases (profiling)')
    ap.add_argument('--paths', default='plain,f16x3,tf32x3,f16x3_raw,tf32x3_raw',
                    help='comma list of plain, tf32x3, f16x3, tf32x3_raw, f16x3_raw (tensor cores in the '
                         'pipelined plan kernels), f16x3_tile, tf32x3_tile, f16x3_k4, tf32x3_k4 (the tile '
                         'kernel), pergate, plain_interp, plain_previous')
    ap.add_argument('--tile-bits', type=int, default=0, help='tile qubits of the tile passes (0 = default)')
    ap.add_argument('--workload', default='34q', choices=['34q', 'batch', 'branch42', 'inner34', 'tensor28'],
                    help='34q: the headline line (with everything else inside it); the others print only '
                         'that secondary workload')
    ap.add_argument('--depth', type=int, default=0, help='override the lattice depth (profiling of smaller cases)')
    ap.add_argument('--pipeline', type=int, default=0, help='plain path: 0 = pipelined persistent kernel, '
                                                            '-1 = one CTA per tile in flight')
    ap.add_argument('--autotune', type=int, default=1, help='plain path: 1 = tile size and per-pass kernel shape '
                                                            'picked by timing on the first call (cached), 0 = defaults')
    ap.add_argument('--no-cpu', action='store_true', help='skip the oracle legs (and the 30q accuracy block)')
    ap.add_argument('--no-extra', action='store_true', help='skip the secondary workloads')
    args = ap.parse_args()

    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    if args.impl == 'reference':
        return run_reference(args, rank, world)
    if args.workload != '34q':
        import torch
        torch.cuda.set_device(local)
        fn = {'batch': lambda: batch_workload(args.steps, args.warmup, ('jit', 'default', 'interp', 'small')),
              'branch42': lambda: branch_workload(args.steps, args.warmup),
              'inner34': lambda: inner_workload(args.steps, args.warmup),
              'tensor28': lambda: tensor_workload(args.steps, args.warmup)}[args.workload]
        line = fn()
        line.update({'workload': args.workload, 'n_gpus': world, 'steps': args.steps, 'warmup': args.warmup})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0

    import numpy as np
    import torch
    from paper_1804_04797_gb300 import inputs, sv

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))

    lat = {34: inputs.C34, 30: inputs.C30, 28: inputs.C28, 16: inputs.C16}.get(args.qubits, inputs.C34)
    if args.depth > 0:
        lat = inputs.Lattice(lat.rows, lat.cols, lat.removed_mask, args.depth, lat.seed)
    n = lat.n_qubits
    gates = sv.sv_generate_circuit(lat)
    stream = torch.cuda.Stream()
    hbm_peak, bf16_peak, peak_kind = _peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(h, steps, warmup, fn):
        for _ in range(warmup):
            fn(h)
        barrier()
        sv.sv_set_profiling(h, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with Clocks(local) as ck:
            ev0.record(stream)
            t0 = time.perf_counter()
            for _ in range(steps):
                fn(h)
            ev1.record(stream)
            barrier()
            wall = time.perf_counter() - t0
        ms = ev0.elapsed_time(ev1)
        prof = sv.sv_get_profile(h)
        launch_ms, _ = sv.sv_get_launch_times(h)
        sv.sv_set_profiling(h, False)
        ms, wall = max_over_ranks([ms, wall], dist, 'cuda')
        # per pass: launch i of every step averaged over the steps
        per = len(launch_ms) // steps if steps else 0
        per_pass = [float(np.mean(launch_ms[i::per])) for i in range(per)] if per else []
        return ms, wall, prof, ck.summary(), per_pass

    def step_device(h):
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, gates)

    results = {}
    bits = np.array(inputs.bitstrings(n, 64, seed=2), dtype=np.uint64)
    known = {'plain': dict(), 'tf32x3': dict(precision=sv.SV_PREC_TF32X3), 'f16x3': dict(precision=sv.SV_PREC_F16X3),
             'tf32x3_raw': dict(precision=sv.SV_PREC_TF32X3, norm_restore=-1),
             'f16x3_raw': dict(precision=sv.SV_PREC_F16X3, norm_restore=-1),
             'f16x3_tile': dict(precision=sv.SV_PREC_F16X3, pipeline=-1),
             'tf32x3_tile': dict(precision=sv.SV_PREC_TF32X3, pipeline=-1),
             'f16x3_k4': dict(precision=sv.SV_PREC_F16X3, fuse_k=4),
             'tf32x3_k4': dict(precision=sv.SV_PREC_TF32X3, fuse_k=4),
             'pergate': dict(precision=sv.SV_PREC_PERGATE), 'plain_interp': dict(jit=-1),
             'plain_previous': dict(pipeline=-1)}
    modes = [p for p in args.paths.split(',') if p in known]
    h = sv.sv_create(n, sv.options(stream=stream.cuda_stream))
    amps_ref = None
    try:
        for name in modes:
            kw = dict(known[name])
            if name == 'plain':
                kw['pipeline'] = args.pipeline
                kw['autotune'] = args.autotune
            # the headline path takes the requested steps; the others fewer (secondary)
            steps, warmup = (args.steps, args.warmup) if name == 'plain' else (min(args.steps, 3), 1)
            if name.endswith('_raw'):
                steps = 1
            try:
                sv.sv_set_options(h, sv.options(stream=stream.cuda_stream, tile_bits=args.tile_bits, **kw))
                ms, wall, prof, clocks, per_pass = timed(h, steps, warmup, step_device)
            except sv.SvError as e:
                results[name] = {'unavailable': str(e)}
                continue
            norm2, sp2 = sv.sv_norm(h)
            amps = sv.sv_get_amplitudes(h, bits)
            if amps_ref is None:
                amps_ref = amps
            agree = float(np.linalg.norm(amps - amps_ref) / np.linalg.norm(amps_ref))
            per_launch_ms = prof.ms / max(prof.launches, 1)
            bytes_per_launch = prof.hbm_bytes / max(prof.launches, 1)
            results[name] = {
                's_per_circuit': ms / 1e3 / steps, 'steps': steps, 'ms_total': ms, 'wall_s': wall,
                'launches': prof.launches, 'kernel_ms': prof.ms, 'kernel_bytes': prof.hbm_bytes,
                'per_launch_ms': per_launch_ms, 'bytes_per_launch': bytes_per_launch,
                'achieved_gbs': bytes_per_launch / (per_launch_ms * 1e-3) / 1e9,
                'norm_err': norm2 - 1.0, 'n_sum_p2': (2.0 ** n) * sp2, 'rel_l2_vs_plain_64amps': agree,
                'clocks': clocks, 'launches_per_step': (prof.launches + prof.other_launches) / steps,
                'plan_kernel_launches': prof.jit_launches, 'per_pass_ms': per_pass,
                # the plan it ran (the autotuner's tile size and fusion width for plain)
                'plan': {'tile_bits': prof.plan_tile_bits, 'stage_qubits': prof.plan_stage_qubits,
                         'passes': prof.plan_passes},
            }

        # end to end through the public API with host buffers: gate list in, amplitudes
        # and norm out, every step
        def step_e2e(hh):
            sv.sv_reset(hh)
            sv.sv_apply_circuit(hh, sv.sv_generate_circuit(lat))
            sv.sv_get_amplitudes(hh, bits)
            sv.sv_norm(hh)
        sv.sv_set_options(h, sv.options(stream=stream.cuda_stream, pipeline=args.pipeline, autotune=args.autotune))
        e2e_steps = max(1, min(args.steps, 3))
        e_ms, e_wall, e_prof, _, _ = timed(h, e2e_steps, 1, step_e2e)
        e2e = {'value': e_wall / e2e_steps, 'unit': UNIT,
               'h2d_bytes_per_step': (e_prof.h2d_bytes + gates.nbytes * e2e_steps) / e2e_steps,
               'd2h_bytes_per_step': e_prof.d2h_bytes / e2e_steps}
    finally:
        sv.sv_destroy(h)

    # secondary workloads (the headline state is freed: the inner product needs two)
    extra = {}
    if not args.no_extra and lat == inputs.C34:
        for key, fn in (('inner34', lambda: inner_workload(1, 1)), ('branch42', lambda: branch_workload(3, 1)),
                        ('tensor28', lambda: tensor_workload(5, 2)),
                        ('batch', lambda: batch_workload(3, 1, ('default', 'small')))):
            try:
                extra[key] = fn()
            except Exception as e:  # reported, not hidden: the headline still prints
                extra[key] = {'unavailable': '%s: %s' % (type(e).__name__, e)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # the oracle's times and the 30-qubit accuracy block against the oracle
    cpu, accuracy = None, None
    if not args.no_cpu:
        times, want = oracle_times()
        accuracy = accuracy_30q(want, stream)
        del want
        o34 = times['34q_d30']
        cpu = {'value': o34['s_per_circuit_all_cores'], 'unit': UNIT, 'cores': times['cores'], 'kind': 'oracle',
               'sample': 'the 30-qubit depth-20 circuit run whole on %d cores (%.1f s); %s'
                         % (times['cores'], times['30q_d20']['s_per_circuit_all_cores'], o34['note']),
               'extrapolated': True, 'scale_factor': o34['scale_factor'], 'measured': times}

    ok = [k for k, r in results.items() if 's_per_circuit' in r and r.get('rel_l2_vs_plain_64amps', 1.0) <= 1e-5]
    best_name = 'plain' if 'plain' in ok else min(ok, key=lambda k: results[k]['s_per_circuit'])
    best = results[best_name]
    value = whole_job_s_per_circuit(best['s_per_circuit'], world)
    kname = {'plain': 'sv_pass (pipelined)' if args.pipeline >= 0 else 'sv_pass', 'plain_previous': 'sv_pass',
             'plain_interp': 'tile_pass_kernel', 'pergate': 'gate1q_kernel/diag_kernel'}
    # the tensor-core paths: matrix stages of the pipelined plan kernels, or the tile kernel
    kernel = kname.get(best_name, 'fused_pass_kernel' if best_name.endswith(('_tile', '_k4'))
                       else 'sv_pass (matrix stages)')
    ratio = TRAFFIC_PER_ALGORITHMIC_BYTE.get(kernel)
    flops = algorithmic_flops_per_amplitude(gates) * 2.0 ** n
    sm_mhz = (best['clocks'] or {}).get('sm_max_mhz') or 2070.0
    lane_peak = SMS * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    line = {
        'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': best['s_per_circuit'] * 1e3, 'higher_is_better': False,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'c64', 'data': 'synthetic',
        'config': {'workload': '34-qubit 6x6-minus-corners lattice circuit, depth 30, seed 0 (478 gates)'
                   if lat == inputs.C34 else '%d-qubit %dx%d lattice circuit, depth %d' % (n, lat.rows, lat.cols,
                                                                                          lat.depth),
                   'state_bytes': 8 * 2 ** n, 'l2': 'state 137 GB >> L2 129 MB, no flush needed',
                   'path': best_name, 'replicas': world},
        'roofline': {'bound': 'hbm', 'kernel': kernel, 'achieved': best['achieved_gbs'], 'peak': hbm_peak,
                     'unit': 'GB/s', 'frac': best['achieved_gbs'] / hbm_peak,
                     'traffic': ratio * best['bytes_per_launch'] if ratio else None, 'peak_kind': peak_kind,
                     'bytes_per_launch': best['bytes_per_launch'], 'per_launch_ms': best['per_launch_ms'],
                     'per_pass_ms': best['per_pass_ms']},
        # the plain kernel's other limit: FP32 lane operations (the gates' arithmetic is
        # additions and multiplications, few of which fuse): algorithmic operations of
        # the circuit over its time, against one operation per FP32 lane per clock
        'roofline_alu': {'bound': 'alu', 'kernel': kernel, 'achieved': flops / best['s_per_circuit'] / 1e12,
                         'peak': lane_peak, 'unit': 'T lane-ops/s',
                         'frac': flops / best['s_per_circuit'] / 1e12 / lane_peak,
                         'ops_per_circuit': flops,
                         'peak_kind': 'instruction-rate bound: 152 SMs x 128 FP32 lanes x max SM clock, one add, '
                                      'multiply or fused multiply-add per lane per clock (an FMA-only mix would '
                                      'count 2 flops per lane-op: %.1f TFLOP/s)' % (2 * lane_peak)},
        'clocks': best['clocks'],
        'e2e': e2e,
        'gpu_launches': int(round(best['launches_per_step'] * args.steps)),
        'cpu_baseline': cpu,
        'paths': results,
    }
    # the tensor-core paths' own roofline: HBM and the tensor pipe. A stage of k qubits
    # with gates in it is, per 2^m-amplitude tile, a real GEMM of 2^(m-k) rows against a
    # 2^(k+1) x 2^(k+1) matrix taken as 3 split products: 3 * 2^(m+k+3) flops.
    tc = {}
    for name in ('f16x3', 'tf32x3', 'f16x3_tile', 'tf32x3_tile', 'f16x3_k4', 'tf32x3_k4'):
        r = results.get(name, {})
        if 's_per_circuit' not in r:
            continue
        kw = dict(known[name])
        summ, *_ = sv.sv_plan(n, gates, sv.options(**kw))
        m, k = 12, kw.get('fuse_k', 0) or 5
        tflops = summ.matrix_stages * 2.0 ** (n - m) * 3 * 2.0 ** (m + k + 3) / r['s_per_circuit'] / 1e12
        kind = name.split('_')[0]
        peak = bf16_peak * TENSOR_RATIO[kind]
        tc[name] = {'hbm': {'achieved': r['achieved_gbs'], 'peak': hbm_peak, 'unit': 'GB/s',
                            'frac': r['achieved_gbs'] / hbm_peak},
                    'tensor': {'achieved': tflops, 'peak': peak, 'unit': 'TFLOP/s', 'frac': tflops / peak,
                               'peak_kind': 'measured bf16 burst x nominal %s/bf16 rate ratio %.3f'
                                            % (kind[:-2], TENSOR_RATIO[kind]),
                               'matrix_stages': summ.matrix_stages, 'k': k}}
    if tc:
        line['roofline_tensor_core_paths'] = tc
    if accuracy is not None:
        line['accuracy_30q'] = accuracy
    if extra:
        line['workloads'] = extra
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == '__main__':
    sys.exit(main())

"""Benchmark: FP64 unknowns*steps/s of the CCF cylinder heat solver on one GB300.

Workload (one bench step): the 128^3 heat problem -- n_r = n_z = n_theta = 128,
alpha = 1, dt = 1e-3, 100 implicit BDF1 steps, T0 = 8 Bessel x sine
eigenmodes with seeded N(0,1) amplitudes, g = seeded smooth CCF coefficients
N(0,1) * 1.25^-(i+j+|k|).  Synthetic inputs; the coefficient fields are
16.8 MB (below the 129 MB L2), so L2 is flushed (a 256 MB write) between timed
steps.  value = N * 100 * K / (sum of the K timed step durations).

Legs: --impl ours (default) times the CUDA path through the C ABI; --impl
reference times the FP64 CPU oracle on the host cores on a bounded sample of
the same workload (slices of the 128^3 field; slices are independent).
Under torchrun each rank runs its own replica (independent problems, weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2206_04827_gb300 import inputs  # noqa: E402

M = N_Z = P = 128
ALPHA, DT, NSTEPS, TOL = 1.0, 1e-3, 100, 1e-14
SEED = 1001
WORKLOAD = 'heat 128^3 (n_r=n_z=n_theta=128), alpha=1, dt=1e-3, 100 BDF1 steps, 8 Bessel x sine eigenmodes + smooth forcing'
METRIC = 'FP64 unknowns*steps/s at <=1e-12 rel err'
UNIT = 'unknowns*steps/s'
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2      # measured: 1192 GFLOP/s at 1980 MHz on 152 SMs


# ----------------------------------------------------------------- CPU oracle leg
def _oracle_worker(args):
    """One oracle run on a subset of slices (runs in a spawned process)."""
    os.environ.setdefault('OMP_NUM_THREADS', '1')
    sys.path.insert(0, ROOT)
    from oracle import heat as oheat
    slices, steps = args
    rng = inputs.rng_for(SEED)
    X0, g = _host_inputs_coeffs(rng)
    t0 = time.perf_counter()
    out = oheat.heat_steps(X0, g, ALPHA, DT, steps, slices=slices)
    dt = time.perf_counter() - t0
    return dt, {s: out[s] for s in slices}


def _host_inputs_coeffs(rng):
    """Smooth seeded coefficients used by the CPU legs (T0 and g drawn from the
    same generator as the GPU leg's g; the CPU legs time throughput only)."""
    X0 = inputs.smooth_coeffs(P, M, N_Z, 1.25, rng)
    g = inputs.smooth_coeffs(P, M, N_Z, 1.25, rng)
    return X0, g


def run_oracle_sample(nslices=16, steps=8, procs=None):
    """Time the oracle as it stands on `nslices` slices x `steps` steps,
    one slice per spawned process (BLAS single-threaded in each)."""
    procs = procs or os.cpu_count() or 1
    sl = [int(s) for s in np.linspace(0, P - 1, nslices).round()]
    ctx = mp.get_context('spawn')
    t0 = time.perf_counter()
    with ctx.Pool(processes=min(procs, nslices)) as pool:
        res = pool.map(_oracle_worker, [([s], steps) for s in sl])
    wall = time.perf_counter() - t0
    out = {}
    for _, d in res:
        out.update(d)
    rate = nslices * M * N_Z * steps / wall
    return rate, wall, min(procs, nslices), sl, out


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,'
                 'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
                 'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap',
                 '--format=csv,noheader,nounits', '-i', str(_local_rank()), '-lms', '100'],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(',')]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        mhz = [float(s[0]) for s in self.samples if s[0].replace('.', '').isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == 'active'})
        return {'sm_mhz': statistics.median(mhz) if mhz else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': reasons, 'samples': len(self.samples)}


def _local_rank():
    return int(os.environ.get('LOCAL_RANK', '0'))


# ----------------------------------------------------------------- flop count
def adi_flops_per_launch(plan, nsteps):
    """Algorithmic FP64 flops of one fused launch (2 per FMA): per item and step,
    the right side (3 + 5 FMA per element), Algorithm 1 (radial sweep 12,
    vertical sweep 8 FMA-class ops per element and iteration; the first
    iteration has no radial apply (-6), the last no vertical apply (-4)) and
    the Dirichlet expansion (3 adds per element)."""
    total = 0.0
    h = P // 2
    for k in range(h + 1):
        pr = k % 2
        J = plan.shifts(1, k, pr)[0]
        nsl = 1 if k in (0, h) else 2
        Mr = (M - 2 - pr + 1) // 2
        Mf = (M - pr + 1) // 2
        for pz in (0, 1):
            Nz = (N_Z - 2 - pz + 1) // 2
            Nf = (N_Z - pz + 1) // 2
            W = nsl * Nz
            per_step = 3 * Mf * W + 5 * Mr * W + (12 * J - 6 + 8 * J - 4) * Mr * W + 1.5 * Mf * nsl * Nf
            total += 2.0 * per_step * nsteps
    return total


# ----------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    if world > 1:
        dist.init_process_group('nccl', init_method='env://')
    torch.cuda.set_device(_local_rank())
    dev = torch.device('cuda', _local_rank())

    # CPU baseline and accuracy sample first (spawned pool before heavy GPU use)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, wall, cores, sl, oracle_out = run_oracle_sample(args.cpu_slices, args.cpu_steps)
        cpu = dict(value=rate, wall=wall, cores=cores, slices=sl, out=oracle_out)

    from paper_2206_04827_gb300 import cyl
    stream = torch.cuda.current_stream(dev)
    plan = cyl.Plan(M, N_Z, P, ALPHA, DT, TOL, poisson=False, heat=True, stream=stream.cuda_stream)
    r, z, th = plan.grid()
    rng = inputs.rng_for(SEED)
    modes = inputs.eigenmode_list(8, rng)
    g_host = inputs.smooth_coeffs(P, M, N_Z, 1.25, rng)
    T0 = torch.empty(P, M, N_Z, dtype=torch.float64, device=dev)
    plan.vals2coeffs(torch.as_tensor(inputs.eigenmode_values(r, z, th, modes), device=dev), T0)
    g = torch.as_tensor(g_host, device=dev)
    T = torch.empty_like(T0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    Nunk = M * N_Z * P

    nst = args.nsteps

    def one_step():
        plan.heat_step(T, g, nst)

    for _ in range(args.warmup):
        T.copy_(T0)
        one_step()
    torch.cuda.synchronize()

    # accuracy: the same run compared with the oracle on the sampled slices
    acc = None
    if cpu is not None:
        rng2 = inputs.rng_for(SEED)
        X0c, gc = _host_inputs_coeffs(rng2)
        Tc = torch.as_tensor(X0c, device=dev)
        plan.heat_step(Tc, torch.as_tensor(gc, device=dev), args.cpu_steps)
        Tc = Tc.cpu().numpy()
        ref = np.stack([cpu['out'][s] for s in cpu['slices']])
        got = np.stack([Tc[s] for s in cpu['slices']])
        acc = float(np.abs(got - ref).max() / np.abs(ref).max())

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler()
    clk.start()
    time.sleep(0.3)
    evs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        T.copy_(T0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    durs = [a.elapsed_time(b) * 1e-3 for a, b in evs]
    t_sum = sum(durs)
    t_max = torch.tensor([t_sum], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    t_sum = float(t_max.item())

    # end to end through the C ABI with pinned host buffers
    T0_h = T0.cpu().pin_memory()
    g_h = g.cpu().pin_memory()
    out_h = torch.empty_like(T0_h).pin_memory()
    e2e = []
    for it in range(args.steps + 1):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        T.copy_(T0_h, non_blocking=True)
        g.copy_(g_h, non_blocking=True)
        one_step()
        out_h.copy_(T, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it > 0:
            e2e.append(e0.elapsed_time(e1) * 1e-3)
    e2e_t = sum(e2e)

    flops = adi_flops_per_launch(plan, nst)
    peak_mhz = clocks['sm_max_mhz'] or 2070.0
    peak = SM_COUNT * FP64_FMA_PER_CLK_PER_SM * 2 * peak_mhz * 1e6
    achieved = flops / (t_sum / args.steps)
    line = {
        'metric': METRIC, 'value': world * Nunk * nst * args.steps / t_sum, 'unit': UNIT,
        'n_gpus': world, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': 1e3 * t_sum / args.steps, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'n_r': M, 'n_z': N_Z, 'n_theta': P, 'time_steps_per_bench_step': nst,
                   'adi_tol': TOL, 'l2': 'flushed between timed steps (256 MB write)',
                   'parallelism': 'replicas' if world > 1 else 'single'},
        'roofline': {'bound': 'alu', 'achieved': achieved / 1e12, 'peak': peak / 1e12, 'unit': 'TFLOP/s',
                     'frac': achieved / peak, 'traffic': None,
                     'peak_basis': '152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock (of derived)',
                     'kernel': 'adi_kernel'},
        'e2e': {'value': world * Nunk * nst * len(e2e) / e2e_t, 'unit': UNIT,
                'h2d_bytes_per_step': int(T0_h.numel() * 8 + g_h.numel() * 8),
                'd2h_bytes_per_step': int(out_h.numel() * 8)},
        'gpu_launches': args.steps,
        'clocks': {k: clocks[k] for k in ('sm_mhz', 'sm_max_mhz', 'reasons')},
        'wall_s': wall,
    }
    if cpu is not None:
        line['cpu_baseline'] = {'value': cpu['value'], 'unit': UNIT, 'cores': cpu['cores'], 'kind': 'oracle',
                                'sample': '%d of %d theta-slices x %d BDF1 steps of the 128^3 problem '
                                          '(QZ Bartels-Stewart per slice, one process per slice)'
                                          % (len(cpu['slices']), P, args.cpu_steps)}
        line['max_rel_err_vs_oracle'] = acc
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    for _ in range(args.warmup):
        run_oracle_sample(args.cpu_slices, 1)
    rates, walls = [], []
    for _ in range(args.steps):
        rate, wall, cores, sl, _ = run_oracle_sample(args.cpu_slices, args.cpu_steps)
        rates.append(rate)
        walls.append(wall)
    value = len(rates) * args.cpu_slices * M * N_Z * args.cpu_steps / sum(walls)
    sample = '%d of %d theta-slices x %d BDF1 steps of the 128^3 problem per bench step' % (
        args.cpu_slices, P, args.cpu_steps)
    print(json.dumps({
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': 0, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': 1e3 * sum(walls) / len(walls), 'higher_is_better': True,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'n_r': M, 'n_z': N_Z, 'n_theta': P},
        'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': cores, 'kind': 'oracle', 'sample': sample},
        'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--cpu-slices', type=int, default=16)
    ap.add_argument('--cpu-steps', type=int, default=10)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--nsteps', type=int, default=NSTEPS,
                    help='BDF1 steps per bench step (100 = the workload; fewer only for profiling)')
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == 'reference':
        run_reference(args)
    else:
        run_ours(args)


if __name__ == '__main__':
    main()

"""Autotuner of the linearized encoding, in place of the paper's DRL agent.

The paper searches the interleavings of the modes' bits (Sec. 3.3.2, Eq. 1)
with a double-DQN agent whose reward is the speedup of the all-mode MTTKRP
over the ALTO encoding (Sec. 3.3.4), using action masking (every episode ends
in a valid order, Sec. 3.4), a reward cache, and elastic early stopping. This
module keeps the search space, the objective and those mechanisms and
replaces the learned policy with a plain search:

* candidates are valid by construction: an order places mode n exactly l(n)
  times (the masking rule);
* seeds: the ALTO order, "mode n on top" orders, block interleaves, the
  longest-mode-first interleave and seeded random interleavings; then local
  search by swapping adjacent bits of different modes in the best order;
* every (order, partition size) is evaluated once (reward cache);
* the search stops when the best speedup has not improved for `patience`
  evaluations, or after `max_evals`;
* per mode, the conflict strategy with the shortest MTTKRP time is kept;
* then, for the best encoding, every mode's kernel plan is searched
  (tune_modes): the conflict strategy, and for the SEGMENTED strategy the
  fiber-factoring depth, the level order of the other modes and the R-tile
  width (R / column passes), each timed and the fastest kept.

`sandbox_reward` reproduces the paper's sandbox mode (reward for reproducing
the ALTO order) and serves as a self-test of the search.
"""
from __future__ import annotations

import math
import random
import time
from dataclasses import dataclass, field

import numpy as np


def bit_budget(dims) -> list[int]:
    out = []
    for I in dims:
        b = 0
        while (1 << b) < int(I):
            b += 1
        out.append(b)
    return out


def alto_order(dims) -> tuple:
    """ALTO default: round robin from b^0 over modes sorted by (l(n), id)."""
    lb = bit_budget(dims)
    rank = sorted(range(len(dims)), key=lambda m: (lb[m], m))
    left = list(lb)
    out = []
    while len(out) < sum(lb):
        for m in rank:
            if left[m]:
                out.append(m)
                left[m] -= 1
    return tuple(out)


def is_valid(order, dims) -> bool:
    lb = bit_budget(dims)
    return len(order) == sum(lb) and all(order.count(m) == lb[m] for m in range(len(dims)))


def mode_on_top(dims, n) -> tuple:
    """All bits of mode n above the ALTO interleave of the other modes (long
    runs of equal i_n in encoded order)."""
    rest = [m for m in alto_order(dims) if m != n]
    return tuple(rest + [n] * bit_budget(dims)[n])


def block_interleave(dims, block: int) -> tuple:
    lb = bit_budget(dims)
    rank = sorted(range(len(dims)), key=lambda m: (lb[m], m))
    left = list(lb)
    out = []
    while len(out) < sum(lb):
        for m in rank:
            take = min(block, left[m])
            out += [m] * take
            left[m] -= take
    return tuple(out)


def longest_first(dims) -> tuple:
    lb = bit_budget(dims)
    rank = sorted(range(len(dims)), key=lambda m: (-lb[m], m))
    left = list(lb)
    out = []
    while len(out) < sum(lb):
        for m in rank:
            if left[m]:
                out.append(m)
                left[m] -= 1
    return tuple(out)


def random_interleave(dims, rng: random.Random) -> tuple:
    base = [m for m, l in enumerate(bit_budget(dims)) for _ in range(l)]
    rng.shuffle(base)
    return tuple(base)


def neighbours(order) -> list[tuple]:
    """Adjacent swaps of bits of different modes (keeps every mode's count)."""
    out = []
    for t in range(len(order) - 1):
        if order[t] != order[t + 1]:
            o = list(order)
            o[t], o[t + 1] = o[t + 1], o[t]
            out.append(tuple(o))
    return out


@dataclass
class Trial:
    order: tuple
    partition_size: int
    seconds: float
    strategies: list
    speedup: float


@dataclass
class TuneResult:
    best: Trial
    baseline: Trial
    trials: list = field(default_factory=list)
    evaluations: int = 0
    cache_hits: int = 0
    stopped_early: bool = False


def tune(dims, evaluate, partition_sizes=(4096,), seed: int = 0, patience: int = 8, max_evals: int = 48,
         n_random: int = 4, verbose: bool = False, baseline_order=None, seeds=None) -> TuneResult:
    """evaluate(order, partition_size) -> (seconds, per-mode strategies).
    Returns the best configuration and the baseline (the ALTO order unless
    baseline_order is given; seeds replaces the default seed orders)."""
    rng = random.Random(seed)
    cache: dict = {}
    res = TuneResult(best=None, baseline=None)

    def run(order, S):
        key = (tuple(order), int(S))
        if key in cache:
            res.cache_hits += 1
            return cache[key]
        assert is_valid(order, dims), order
        secs, strat = evaluate(tuple(order), int(S))
        res.evaluations += 1
        base = res.baseline.seconds if res.baseline else secs
        tr = Trial(tuple(order), int(S), secs, list(strat), base / secs if secs > 0 else 0.0)
        cache[key] = tr
        res.trials.append(tr)
        if verbose:
            print(f"  eval {res.evaluations}: S={S} speedup {tr.speedup:.3f} ({secs * 1e3:.3f} ms)", flush=True)
        return tr

    res.baseline = run(tuple(baseline_order) if baseline_order is not None else alto_order(dims),
                       partition_sizes[0])
    res.best = res.baseline
    if seeds is None:
        seeds = [alto_order(dims)] + [mode_on_top(dims, n) for n in range(len(dims))]
        seeds += [block_interleave(dims, b) for b in (2, 4)] + [longest_first(dims)]
        seeds += [random_interleave(dims, rng) for _ in range(n_random)]
    seeds = [tuple(o) for o in seeds]
    since = 0
    expanded = set()
    queue = [(o, S) for o in dict.fromkeys(seeds) for S in partition_sizes]
    while res.evaluations < max_evals:
        if not queue:  # local search around the best order found so far
            key = (res.best.order, res.best.partition_size)
            if key in expanded:
                break
            expanded.add(key)
            queue = [(o, res.best.partition_size) for o in neighbours(res.best.order)]
            continue
        order, S = queue.pop(0)
        before = res.evaluations
        tr = run(order, S)
        if res.evaluations == before:
            continue
        if tr.seconds < res.best.seconds:
            res.best = tr
            since = 0
            expanded.add((tr.order, tr.partition_size))
            queue = [(o, tr.partition_size) for o in neighbours(tr.order)] + queue
        else:
            since += 1
        if since >= patience:
            res.stopped_early = True
            break
    return res


def kendall_distance(order, target) -> int:
    """Adjacent swaps needed to turn `order` into `target` (same multiset):
    the k-th occurrence of a mode in one is matched with its k-th occurrence
    in the other and the inversions of that matching are counted."""
    seen: dict = {}
    where: dict = {}
    for t, m in enumerate(target):
        where.setdefault(m, []).append(t)
    mapped = []
    for m in order:
        k = seen.get(m, 0)
        seen[m] = k + 1
        mapped.append(where[m][k])
    return sum(1 for i in range(len(mapped)) for j in range(i + 1, len(mapped)) if mapped[i] > mapped[j])


def sandbox_reward(dims):
    """The paper's sandbox mode: no benchmark, the reward is reproducing the
    ALTO order. Returned as an evaluator whose "time" is 1 + the number of
    adjacent swaps still separating the order from ALTO's."""
    target = alto_order(dims)

    def evaluate(order, S):
        return 1.0 + kendall_distance(order, target), ["sandbox"] * len(dims)

    return evaluate


def gpu_evaluator(coords_dev, vals_dev, dims, R: int, factor_dtype: str, factors, reps: int = 3,
                  strategies=(1, 2, 3)):
    """Times the all-mode MTTKRP of an encoding on the GPU (CUDA events on the
    current stream); per mode the fastest conflict strategy is kept."""
    import torch

    from . import relate as rl

    dev = coords_dev.device
    acc = torch.float64 if factor_dtype == "f64" else torch.float32
    outs = [torch.empty((int(d), R), dtype=acc, device=dev) for d in dims]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def evaluate(order, S):
        h = rl.relate_encode(coords_dev, vals_dev, dims, bit_order=np.array(order, dtype=np.int8),
                             partition_size=S, factor_dtype=factor_dtype)
        total, chosen = 0.0, []
        for n in range(len(dims)):
            best = (math.inf, 0)
            for strat in strategies:
                if strat == 3 and int(dims[n]) * R * (8 if factor_dtype == "f64" else 4) > 32 * 1024:
                    continue
                rl.relate_set_conflict(h, n, strat)
                ts = []
                for r in range(reps + 1):
                    flush.fill_(float(r))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    rl.relate_mttkrp(h, n, factors, R, outs[n])
                    e1.record()
                    torch.cuda.synchronize()
                    if r:
                        ts.append(e0.elapsed_time(e1) / 1e3)
                t = float(np.median(ts))
                if t < best[0]:
                    best = (t, strat)
            total += best[0]
            chosen.append(best[1])
        h.close()
        return total, chosen

    return evaluate


@dataclass
class ModeConfig:
    strategy: int            # relate_conflict_t (1 atomic, 2 segmented, 3 privatized)
    depth: int = 0           # fiber-factoring levels (SEGMENTED, 3..5 modes)
    level: tuple | None = None  # order of the other modes (None = AUTO)
    col_passes: int = 1      # R-tile width = R / col_passes
    kr: int = 0              # FP64: fuse the innermost two modes' Khatri-Rao pair (relate_set_mode_kr)

    def as_dict(self) -> dict:
        return {"strategy": self.strategy, "depth": self.depth,
                "level": list(self.level) if self.level is not None else None, "col_passes": self.col_passes,
                "kr": self.kr}


# The library's limits of a Khatri-Rao table: rows below 2^32 and 16 GiB of FP64.
KR_MAX_BYTES = 16 << 30


def kr_fits(dims, level, depth, R) -> bool:
    """The pair (level[depth - 1], level[depth]) of an FP64 plan can be fused."""
    if depth < 2 or depth != len(level) - 1 or R % 2:  # one unfactored slot
        return False
    rows = int(dims[level[depth - 1]]) * int(dims[level[depth]])
    return rows < 2 ** 32 and rows * R * 8 <= KR_MAX_BYTES


def mode_configs(dims, mode: int, R: int, factor_dtype: str) -> list[ModeConfig]:
    """The kernel plans tune_modes tries for one mode: ATOMIC; PRIVATIZED when
    the output fits a block's shared memory; SEGMENTED flat and, for 3 to 5
    modes, at every fiber-factoring depth with the other modes longest first
    or shortest first, with the whole row or half of it per pass (R-tile);
    FP64 plans of depth N - 2 also with their innermost Khatri-Rao pair fused
    where its table fits."""
    N = len(dims)
    accb = 8 if factor_dtype == "f64" else 4
    vec = 2 if factor_dtype == "f64" else 4
    out = [ModeConfig(1), ModeConfig(2)]
    if int(dims[mode]) * R * accb <= 32 * 1024:
        out.append(ModeConfig(3))
    if 3 <= N <= 5:
        others = [k for k in range(N) if k != mode]
        longest = tuple(sorted(others, key=lambda k: (-int(dims[k]), k)))
        shortest = tuple(sorted(others, key=lambda k: (int(dims[k]), k)))
        passes = [1] + ([2] if R % 2 == 0 and (R // 2) % vec == 0 else [])
        for depth in range(1, N - 1):
            for level in dict.fromkeys((longest, shortest)):
                krs = [0, 1] if factor_dtype == "f64" and kr_fits(dims, level, depth, R) else [0]
                for p in passes:
                    for kr in krs:
                        out.append(ModeConfig(2, depth, level, p, kr))
    return out


def apply_config(rl, h, mode: int, cfg: ModeConfig) -> None:
    rl.relate_set_conflict(h, mode, cfg.strategy)
    rl.relate_set_mode_plan(h, mode, cfg.depth if cfg.strategy == 2 else 0,
                            list(cfg.level) if cfg.level is not None else None, cfg.col_passes)
    rl.relate_set_mode_kr(h, mode, cfg.kr)


def tune_modes(h, dims, R: int, factor_dtype: str, factors, reps: int = 3, verbose: bool = False, stream=None,
               flush_l2: bool = True):
    """Per mode, times every plan of mode_configs on the encoded tensor (CUDA
    events on `stream`, default the current stream; L2 flushed between
    launches unless flush_l2 is False) and keeps the fastest; the handle is
    left with the chosen plans. Only `stream` is synchronised, so a serving
    worker can tune while other streams run. Returns [(ModeConfig, seconds,
    AUTO seconds)]."""
    import torch

    from . import relate as rl

    dev = factors[0].device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    acc = torch.float64 if factor_dtype == "f64" else torch.float32
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev) if flush_l2 else None
    chosen = []
    for n in range(len(dims)):
        out = torch.empty((int(dims[n]), R), dtype=acc, device=dev)

        def time_mode():
            ts = []
            with torch.cuda.stream(st):
                for r in range(reps + 1):
                    if flush is not None:
                        flush.fill_(float(r))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    rl.relate_mttkrp(h, n, factors, R, out, st)
                    e1.record(st)
                    st.synchronize()
                    if r:
                        ts.append(e0.elapsed_time(e1) / 1e3)
            return float(np.median(ts))

        rl.relate_set_conflict(h, n, 0)
        rl.relate_set_mode_plan(h, n, -1, None, 0)
        rl.relate_set_mode_kr(h, n, -1)
        t_auto = time_mode()
        best = (math.inf, None)
        for cfg in mode_configs(dims, n, R, factor_dtype):
            apply_config(rl, h, n, cfg)
            t = time_mode()
            if verbose:
                print(f"  mode {n} {cfg.as_dict()}: {t * 1e3:.3f} ms", flush=True)
            if t < best[0]:
                best = (t, cfg)
        apply_config(rl, h, n, best[1])
        chosen.append((best[1], best[0], t_auto))
    return chosen


def main(argv=None):
    """Tunes one named synthetic workload on cuda:0 and prints a JSON line."""
    import argparse
    import json
    import os
    import sys

    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="zipf4d-5Mx1Mx100Kx24-150M")
    ap.add_argument("--nnz", type=int, default=0)
    ap.add_argument("--factor-dtype", default=None)
    ap.add_argument("--max-evals", type=int, default=32)
    ap.add_argument("--patience", type=int, default=8)
    ap.add_argument("--shuffle", action="store_true")
    args = ap.parse_args(argv)
    w = synth.WORKLOADS[args.workload]
    spec = w["spec"]
    if args.nnz:
        spec = synth.scaled(spec, args.nnz)
    spec.shuffle = args.shuffle
    R = w["R"]
    fdt = args.factor_dtype or w["factor_dtype"]
    c, v = synth.make_tensor(spec)
    dev = torch.device("cuda:0")
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[fdt]
    dc = torch.from_numpy(c).to(dev)
    dv = torch.from_numpy(v).to(dev)
    fs = [torch.from_numpy(f).to(dev).to(tdt).contiguous() for f in synth.init_factors(spec.dims, R, seed=0)]
    t0 = time.time()
    res = tune(spec.dims, gpu_evaluator(dc, dv, spec.dims, R, fdt, fs), partition_sizes=(4096, 8192, 2048),
               max_evals=args.max_evals, patience=args.patience)
    # the kernel plan of every mode on the best encoding
    from . import relate as rl
    h = rl.relate_encode(dc, dv, spec.dims, bit_order=np.array(res.best.order, dtype=np.int8),
                         partition_size=res.best.partition_size, factor_dtype=fdt)
    modes = tune_modes(h, spec.dims, R, fdt, fs)
    h.close()
    line = {"workload": spec.name, "nnz": spec.nnz, "shuffled": args.shuffle, "R": R, "factor_dtype": fdt,
            "mode_plans": [dict(c.as_dict(), rtile=R // c.col_passes, ms=t * 1e3, auto_ms=ta * 1e3)
                           for c, t, ta in modes],
            "tuned_total_ms": sum(t for _, t, _ in modes) * 1e3, "auto_total_ms": sum(ta for _, _, ta in modes) * 1e3,
            "alto_ms": res.baseline.seconds * 1e3, "best_ms": res.best.seconds * 1e3,
            "speedup_over_alto": res.baseline.seconds / res.best.seconds,
            "best_order": list(res.best.order), "best_partition_size": res.best.partition_size,
            "best_strategies": res.best.strategies, "alto_strategies": res.baseline.strategies,
            "evaluations": res.evaluations, "cache_hits": res.cache_hits, "stopped_early": res.stopped_early,
            "tuning_seconds": time.time() - t0}
    print(json.dumps(line), flush=True)
    return line


if __name__ == "__main__":
    main()

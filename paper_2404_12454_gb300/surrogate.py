"""Surrogate-guided search over the decomposition's free parameters (Sec. 6 asks which
overlap factor and number of beamlets reproduce the Airy pattern best).

Every candidate (N beamlets across, overlap factor, waist ratio) is judged by a real GBD
evaluation: a batched sweep on the GPU (gbd_sweep_*), which returns the RMS error of the
PSF against the analytic Airy amplitude.  The surrogate is the library's MLP (gbd_mlp_*,
trained on the GPU by its own training kernel: forward, backward and Adam in one launch
per fit) fitted to log10 of those scores; each round it ranks a random candidate pool, the
best `per_round` candidates are verified by a sweep and appended to the data, and the
network is refitted.  Plain grid
search (21 OF x 12 WR x 5 N = 1,260 evaluations) is the reference and the fallback, and
random search at an equal budget is the ablation without the network.

Host-side logic only (data bookkeeping, candidate draws, selection); the evaluations and
the network run in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import gbd
from . import workloads as W

# Fixed affine standardisation of the inputs over the search box: OF in [1, 3],
# WR in [0.8, 3], log2 N in [4, 8] map to roughly [-1.7, 1.7].
_CENTER = np.array([2.0, 1.9, 6.0])
_SCALE = np.array([0.577, 0.635, 1.414])


def standardize(params: Sequence[Tuple[int, float, float]]) -> np.ndarray:
    a = np.array([(p[1], p[2], math.log2(p[0])) for p in params], dtype=np.float64)
    return ((a - _CENTER) / _SCALE).astype(np.float32)


def evaluate(params: Sequence[Tuple[int, float, float]], shape=None, optics=None) -> np.ndarray:
    """Airy scores of parameter sets (n_across, OF, WR), via the GPU.  `optics` maps a list
    of parameter sets to the sweep description that evaluates them (default: the thin-lens
    sweep optics, workloads.sweep_from_params; workloads.telescope_sweep_from_params traces
    the App. B telescope instead)."""
    make = optics if optics is not None else W.sweep_from_params
    plan = gbd.sweep_plan(make(list(params)), shape=shape)
    try:
        s = plan.run().cpu().numpy().copy()
        gbd.gbd_sync()
    finally:
        plan.close()
    return s


class MLP:
    """The library's surrogate network with FP32 master weights, BF16 working weights and
    Adam moments in device memory."""

    def __init__(self, seed: int = W.SEED_SURROGATE, device: str = "cuda"):
        import torch
        rng = np.random.default_rng(seed)
        parts = []
        for out_f, in_f in ((128, 3), (128, 128), (128, 128), (128, 128), (1, 128)):
            bound = 1.0 / math.sqrt(in_f)
            parts.append(rng.uniform(-bound, bound, size=out_f * in_f))
            parts.append(rng.uniform(-bound, bound, size=out_f))
        p = np.concatenate(parts).astype(np.float32)
        assert p.size == gbd.MLP_PARAMS
        self.device = device
        self.master = torch.tensor(p, device=device)
        self.weights = torch.empty(p.size, dtype=torch.int16, device=device)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.step = 0
        gbd.gbd_mlp_pack(self.master, self.weights)

    def fit(self, x: np.ndarray, y: np.ndarray, steps: int = 400, lr: float = 2e-3) -> float:
        """Full-batch Adam steps on (x, y); returns the last loss."""
        import torch
        xt = torch.tensor(np.ascontiguousarray(x, dtype=np.float32), device=self.device)
        yt = torch.tensor(np.ascontiguousarray(y, dtype=np.float32), device=self.device)
        ws = torch.empty(gbd.gbd_mlp_workspace_bytes(xt.shape[0]), dtype=torch.uint8,
                         device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        if steps > 0:
            gbd.gbd_mlp_train(self.master, self.weights, self.m, self.v, xt, yt, lr, 0.9, 0.999,
                              1e-8, self.step + 1, steps, loss, ws)
            self.step += steps
        return float(loss.item())

    def predict(self, x: np.ndarray) -> np.ndarray:
        import torch
        xt = torch.tensor(np.ascontiguousarray(x, dtype=np.float32), device=self.device)
        y = torch.empty(xt.shape[0], dtype=torch.float32, device=self.device)
        gbd.gbd_mlp_forward(self.weights, xt, y)
        return y.cpu().numpy()

    def state(self) -> dict:
        return {"master": self.master.cpu().numpy(), "m": self.m.cpu().numpy(),
                "v": self.v.cpu().numpy(), "step": self.step}


@dataclasses.dataclass
class SearchResult:
    params: List[Tuple[int, float, float]]
    scores: List[float]
    best_curve: List[Tuple[int, float]]  # (evaluations so far, best score so far)

    @property
    def best(self) -> Tuple[Tuple[int, float, float], float]:
        k = int(np.argmin(self.scores))
        return self.params[k], self.scores[k]

    def evals_to_reach(self, target: float) -> Optional[int]:
        for n, s in self.best_curve:
            if s <= target:
                return n
        return None


def _curve(scores: Sequence[float], steps: Sequence[int]) -> List[Tuple[int, float]]:
    out, best, n = [], math.inf, 0
    for k in steps:
        best = min(best, float(np.min(scores[n:n + k])))
        n += k
        out.append((n, best))
    return out


def grid_search(optics=None) -> SearchResult:
    """The regular reference grid: 21 OF x 12 WR x 5 N, one batched sweep."""
    sw = W.grid_sweep()
    params = [(sw.n_across[k], sw.overlap_factor[k], sw.waist_ratio[k]) for k in range(sw.n_instances)]
    s = evaluate(params, optics=optics)
    return SearchResult(params, list(s), [(len(params), float(np.min(s)))])


def random_candidates(n: int, rng: np.random.Generator) -> List[Tuple[int, float, float]]:
    of = rng.uniform(1.0, 3.0, size=n)
    wr = rng.uniform(0.8, 3.0, size=n)
    N = rng.choice(np.asarray(W.SWEEP_N_ACROSS), size=n)
    return [(int(a), float(b), float(c)) for a, b, c in zip(N, of, wr)]


def random_search(budget: int, batch: int = 64, seed: int = W.SEED_SURROGATE + 1,
                  optics=None) -> SearchResult:
    """`budget` uniform draws over the search box, drawn and counted `batch` at a time (the
    first batch equals a surrogate search's initial sample of that size and seed)."""
    rng = np.random.default_rng(seed)
    steps = [batch] * (budget // batch) + ([budget % batch] if budget % batch else [])
    params = []
    for k in steps:
        params += random_candidates(k, rng)
    s = evaluate(params, optics=optics)
    return SearchResult(params, list(s), _curve(s, steps))


def surrogate_search(rounds: int = 8, per_round: int = 64, n_init: int = 128, pool: int = 16384,
                     fit_steps: int = 400, seed: int = W.SEED_SURROGATE,
                     checkpoint: Optional[str] = None, target: Optional[float] = None,
                     min_rounds: int = 1, init_seed: Optional[int] = None,
                     optics=None) -> SearchResult:
    """Seeded initial sample (the first n_init instances of the 1024-instance sweep, or
    n_init random candidates drawn with `init_seed`), then rounds of fit -> rank a random
    pool -> verify the best per_round candidates.  After `min_rounds` rounds it stops early
    once the best verified score reaches `target` (if given).  With `checkpoint`, the data
    and the network are saved after every round and a run resumes from them.  `optics` as
    in `evaluate`."""
    if init_seed is None:
        sw = W.sweep()
        params = [(sw.n_across[k], sw.overlap_factor[k], sw.waist_ratio[k])
                  for k in range(n_init)]
    else:
        params = random_candidates(n_init, np.random.default_rng(init_seed))
    start_round = 0
    net = MLP(seed)
    if checkpoint and os.path.exists(checkpoint):
        ck = np.load(checkpoint, allow_pickle=False)
        params = [(int(a), float(b), float(c)) for a, b, c in ck["params"]]
        scores = list(ck["scores"])
        steps = list(ck["steps"])
        start_round = int(ck["round"])
        import torch
        net.master.copy_(torch.tensor(ck["master"]))
        net.m.copy_(torch.tensor(ck["m"]))
        net.v.copy_(torch.tensor(ck["v"]))
        net.step = int(ck["step"])
        gbd.gbd_mlp_pack(net.master, net.weights)
    else:
        scores = list(evaluate(params, optics=optics))
        steps = [n_init]
    rng = np.random.default_rng(seed + 1000)
    for _ in range(start_round):  # keep the candidate stream identical on resume
        random_candidates(pool, rng)
    for r in range(start_round, rounds):
        if target is not None and r >= min_rounds and min(scores) <= target:
            break
        y = np.log10(np.asarray(scores))
        mu, sd = float(y.mean()), float(y.std() + 1e-12)
        net.fit(standardize(params), (y - mu) / sd, steps=fit_steps)
        cand = random_candidates(pool, rng)
        pred = net.predict(standardize(cand))
        order = np.argsort(pred, kind="stable")
        chosen = [cand[k] for k in order[:per_round]]
        s = evaluate(chosen, optics=optics)
        params += chosen
        scores += list(s)
        steps.append(len(chosen))
        if checkpoint:
            st = net.state()
            np.savez(checkpoint, params=np.array(params, dtype=np.float64),
                     scores=np.array(scores), steps=np.array(steps), round=r + 1, **st)
    return SearchResult(params, scores, _curve(np.asarray(scores), steps))


def compare_with_random(target: float, seeds: Sequence[int], n_init: int = 32,
                        per_round: int = 32, budget: int = 1260, optics=None) -> dict:
    """Evaluations each method needs to come within `target`, per seed: the surrogate
    search from n_init random draws (then rounds of per_round proposals), and random search
    drawing per_round candidates at a time, both capped at `budget` evaluations (None when
    the cap is hit first).  Both start from the same seeded draw of n_init candidates."""
    out = {"seeds": list(seeds), "surrogate": [], "random": []}
    rounds = (budget - n_init) // per_round
    for sd in seeds:
        sur = surrogate_search(rounds=rounds, per_round=per_round, n_init=n_init,
                               seed=W.SEED_SURROGATE + sd, target=target, min_rounds=0,
                               init_seed=sd, optics=optics)
        out["surrogate"].append(sur.evals_to_reach(target))
        rnd = random_search(budget=budget, batch=n_init if n_init == per_round else per_round,
                            seed=sd, optics=optics)
        out["random"].append(rnd.evals_to_reach(target))
    return out


def time_training(batch: int = 1024, steps: int = 100, seed: int = 0) -> float:
    """Microseconds per full-batch training step of a fresh network on `batch` synthetic
    samples (inputs ~ N(0, 1), target = first input), after 5 untimed steps: wall time of
    one MLP.fit call (host copies of the data, workspace allocation, the loss read back)."""
    import time

    import torch
    net = MLP()
    xs = np.random.default_rng(seed).normal(size=(batch, 3)).astype(np.float32)
    net.fit(xs, xs[:, 0], steps=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.fit(xs, xs[:, 0], steps=steps)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps * 1e6


def time_training_device(batch: int = 1024, steps: int = 100, seed: int = 0) -> float:
    """Microseconds per training step on the device: CUDA events on the current stream
    around one gbd_mlp_train call of `steps` steps (data and workspace resident), after a
    5-step warm-up call."""
    import torch
    net = MLP()
    rng = np.random.default_rng(seed)
    xt = torch.tensor(rng.normal(size=(batch, 3)).astype(np.float32), device=net.device)
    yt = xt[:, 0].contiguous()
    ws = torch.empty(gbd.gbd_mlp_workspace_bytes(batch), dtype=torch.uint8, device=net.device)
    loss = torch.zeros(1, dtype=torch.float32, device=net.device)
    gbd.gbd_mlp_train(net.master, net.weights, net.m, net.v, xt, yt, 2e-3, 0.9, 0.999, 1e-8, 1,
                      5, loss, ws)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    gbd.gbd_mlp_train(net.master, net.weights, net.m, net.v, xt, yt, 2e-3, 0.9, 0.999, 1e-8, 6,
                      steps, loss, ws)
    stop.record()
    gbd.gbd_sync()
    return start.elapsed_time(stop) / steps * 1e3


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="time the surrogate network's training step")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=100)
    a = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps({"batch": a.batch, "steps": a.steps,
                      "us_per_step": time_training(a.batch, a.steps),
                      "device_us_per_step": time_training_device(a.batch, a.steps)}))

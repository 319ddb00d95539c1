"""Learned scheduling for batched alignment: wave logs -> trained cost model -> batch plan.

The network itself (features, forward, backward, Adam) runs in the library's
kernels (gwfa_model_*); this module only moves tensors between those calls:

* collect(): run a batch with the engine and keep, per query, the raw features
  and the targets log1p(edit distance, peak |Q|, visited diagonals, cells) --
  the work counters the alignment kernels report;
* fit(): set the normalisation from the training set, then train on the GPU;
* plan(): predictions -> (order, n_huge, n_wide) for gwfa_align_batch[_device]:
  longest predicted work first, predicted hash overflows straight onto the
  large-slab classes (huge, wide) that run beside tier 0.  The plain scheduler is
  the input order or length order, with every query starting in tier 0.
"""
from __future__ import annotations

import numpy as np

from . import CostModel, DeviceBatch, Engine, Graph, MODEL_TARGETS

FIELDS = ("edit_distance", "peak_frontier", "visited", "cells")


def targets_of(results: np.ndarray) -> np.ndarray:
    """log1p work counters of each query (n x 4, float32)."""
    return np.stack([np.log1p(results[f].astype(np.float64)) for f in FIELDS], axis=1).astype(np.float32)


def collect(model: CostModel, engine: Engine, queries, order=None):
    """(features, targets, results) of one batch; features and targets as device tensors,
    restricted to the queries that aligned."""
    import torch
    batch = DeviceBatch(queries, device=engine.graph.device, order=order)
    batch.run(engine)
    res = batch.results()
    feat = model.features(batch)
    torch.cuda.synchronize()
    ok = np.nonzero(res["status"] == 0)[0]
    idx = torch.from_numpy(ok.astype(np.int64)).to(feat.device)
    tgt = torch.from_numpy(targets_of(res[ok])).to(feat.device)
    return feat.index_select(0, idx).contiguous(), tgt, res


def fit(model: CostModel, feat, target, steps: int = 1500, batch: int = 512, lr: float = 3e-3,
        seed: int = 7):
    """Normalise from the training set, then train; returns the per-step losses."""
    f = feat.double()
    t = target.double()
    fmean = f.mean(0).cpu().numpy()
    fstd = f.std(0).clamp_min(1e-3).cpu().numpy()
    tmean = t.mean(0).cpu().numpy()
    tstd = t.std(0).clamp_min(1e-3).cpu().numpy()
    model.set_normalization(fmean, fstd, tmean, tstd)
    return model.train(feat, target, steps=steps, batch=batch, lr=lr, seed=seed)


def r2(pred: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Coefficient of determination per target column."""
    ss_res = ((pred - target) ** 2).sum(0)
    ss_tot = ((target - target.mean(0)) ** 2).sum(0)
    return 1.0 - ss_res / np.maximum(ss_tot, 1e-12)


def transfer(src: CostModel, dst: CostModel):
    """Copy weights and normalisation (they do not depend on the graph)."""
    dst.params = src.params
    dst.set_normalization(*src.norm)


def save(model: CostModel, path: str):
    """Weights and normalisation to `path` (the library's gwfa_model_save format)."""
    model.save(path)


def load_into(model: CostModel, path: str):
    """Weights and normalisation from a file written by save (gwfa_model_load)."""
    model.load(path)


def capacities(config) -> tuple[int, int]:
    """(tier-0 tiles, wide-class tiles) a query may fill before it overflows: the
    hash tables' 0.75 load limit; wide 0 when the engine has no huge class."""
    tier0 = int(0.75 * (1 << config.tiers[0].log2_tiles))
    wide = int(0.75 * (1 << config.wide.log2_tiles)) if config.huge.ctas else 0
    return tier0, wide


def plan(model: CostModel, batch: DeviceBatch, engine: Engine):
    """(order, n_huge, n_wide) for `batch` from the model's predictions."""
    from . import plan_schedule
    pred = model.predict(model.features(batch)).cpu().numpy()
    return plan_schedule(pred, *capacities(engine.config))


def time_coeffs(results: np.ndarray) -> tuple[float, float]:
    """Least-squares fit of a query's CTA time: t_us ~ a * scores + b * cells (both >= 0).
    The per-score term is the latency of one score's phases, the per-cell term the
    work; their ratio decides how many CTAs a set of queries needs."""
    ok = results["status"] == 0
    A = np.stack([results["n_scores"][ok].astype(np.float64), results["cells"][ok].astype(np.float64)], 1)
    y = results["device_us"][ok].astype(np.float64)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(max(coef[0], 0.0)), float(max(coef[1], 0.0))


def predicted_time(pred: np.ndarray, coeffs: tuple[float, float] | None) -> np.ndarray:
    d = np.expm1(pred[:, 0].astype(np.float64))
    cells = np.expm1(pred[:, 3].astype(np.float64))
    if coeffs is None:
        return cells
    return coeffs[0] * (d + 1.0) + coeffs[1] * cells


def lpt_max_load(times: np.ndarray, ctas: int) -> float:
    """Largest CTA load when `times` are handed out longest first to `ctas` CTAs, each
    taking the next one when it becomes free (the work queue's behaviour)."""
    import heapq
    loads = [0.0] * max(ctas, 1)
    for x in sorted((float(v) for v in times), reverse=True):
        heapq.heappush(loads, heapq.heappop(loads) + x)
    return max(loads)


def wide_ctas(pred: np.ndarray, order: np.ndarray, n_wide: int, total_ctas: int,
              coeffs: tuple[float, float] | None = None, first: int = 0) -> int:
    """CTAs for a large-slab class holding queue positions [first, first + n_wide):
    its share of the predicted CTA time (or of the predicted cells without time
    coefficients) times the CTAs that fit on the GPU -- raised until the class's own
    longest-first packing ends within the batch's predicted time (the larger of the
    total time spread over every CTA and the longest single query), because a class
    with too few CTAs turns its heaviest queries into a tail; one per query when the
    class is small; at least one, at most one per query of the class."""
    if n_wide == 0:
        return 0
    if n_wide * 8 <= total_ctas:
        # a few heavy queries: one CTA each costs at most an eighth of the GPU for the
        # time the lighter ones keep it busy, and no heavy query waits for another
        return int(n_wide)
    t = predicted_time(pred, coeffs)
    tw = t[order[first:first + n_wide]]
    share = tw.sum() / max(t.sum(), 1e-9)
    c = int(min(n_wide, max(1, round(total_ctas * share))))
    bound = max(t.sum() / max(total_ctas, 1), float(tw.max())) * 1.05
    while c < n_wide and lpt_max_load(tw, c) > bound:
        c = min(n_wide, c + max(1, c // 8))
    return c


def spearman(a: np.ndarray, b: np.ndarray) -> float:
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    return float(np.corrcoef(ra, rb)[0, 1])


__all__ = ["collect", "fit", "plan", "r2", "save", "load_into", "transfer", "targets_of", "spearman",
           "time_coeffs", "predicted_time", "wide_ctas", "lpt_max_load", "capacities", "MODEL_TARGETS", "Graph"]

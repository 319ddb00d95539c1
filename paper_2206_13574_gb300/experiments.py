"""Measurements on the workloads beside the benchmark's (run on a GPU).

    python -m paper_2206_13574_gb300.experiments config3     # cyclic graph: exact vs lag-pruned
    python -m paper_2206_13574_gb300.experiments scheduler   # large graph: learned vs plain scheduling
    python -m paper_2206_13574_gb300.experiments scheduler100k   # the same at 100k queries (two plans)
    python -m paper_2206_13574_gb300.experiments serving     # server vs one-query-at-a-time
    python -m paper_2206_13574_gb300.experiments serving5    # the same on the 50 Mb graph (config 5)

Each prints one JSON line.  Inputs are the seeded synthetic workloads of synth.py.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np


def _timed_run(engine, batch, reps=1, **kw):
    import torch
    st = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        batch.run(engine, **kw)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def config3(n_pruned: int = 2000, n_exact: int = 200, a_diff: int = 1000) -> dict:
    """Cyclic graph with tandem-repeat loops, 50 kb queries at 8% errors: the lag-pruned
    distances (upper bounds) against exact ones on a subset, with both timings."""
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import synth
    import torch
    g, qs = synth.make_config(3, n_queries=n_pruned)
    graph = gw.Graph.from_synth(g)
    order = np.argsort(-qs.lengths(), kind="stable").astype(np.uint32)
    bp = gw.DeviceBatch(qs, order=order)
    engp = gw.Engine(graph, prune=True)
    bp.run(engp, max_lag=a_diff)
    t_pr = _timed_run(engp, bp, max_lag=a_diff)
    pr = bp.results()
    engp.close()
    sub = qs.subset(np.arange(n_exact))
    be = gw.DeviceBatch(sub)
    cfg = gw.default_config(graph)
    cfg.tiers[0].ctas, cfg.tiers[0].log2_tiles = 304, 20
    cfg.tiers[1].ctas, cfg.tiers[1].log2_tiles = 38, 22
    cfg.tiers[2].ctas, cfg.tiers[2].log2_tiles = 4, 24
    enge = gw.Engine(graph, config=cfg)
    t_ex = _timed_run(enge, be)
    ex = be.results()
    enge.close()
    torch.cuda.synchronize()
    # the same pruned run with H~ bounded to the lag window, on slabs 16x smaller
    cfgb = gw.default_config(graph, prune=True)
    slab_small = cfgb.tiers[0].log2_tiles - 4
    cfgb.tiers[0].log2_tiles = slab_small
    engb = gw.Engine(graph, prune=True, config=cfgb)
    bp.run(engb, max_lag=a_diff, evict_lag=a_diff, evict_every=64)
    t_b = _timed_run(engb, bp, max_lag=a_diff, evict_lag=a_diff, evict_every=64)
    bd = bp.results()
    bounded = {"slab_log2_tiles": slab_small, "evict_lag": a_diff, "evict_every": 64, "s": t_b,
               "gbp_per_s": float(qs.lengths()[bd["status"] == 0].sum()) / t_b / 1e9,
               "engine_bytes": engb.device_bytes, "tier0_overflows": int(engb.last_retries()[0]),
               "evicted": int(bd["evicted"].sum()), "cells": int(bd["cells"].sum()),
               "ok": int((bd["status"] == 0).sum())}
    engb.close()
    free_retries = None
    engp2 = gw.Engine(graph, prune=True)
    bp.run(engp2, max_lag=a_diff)
    free_retries = int(engp2.last_retries()[0])
    free_bytes = engp2.device_bytes
    engp2.close()
    prs = pr[:n_exact]
    ok = (ex["status"] == 0) & (prs["status"] == 0)
    return {"workload": "config3: 1 Mb cyclic graph (tandem-repeat loops), 50 kb queries, 8% errors",
            "pruned": {"queries": n_pruned, "a_diff": a_diff, "s": t_pr,
                       "gbp_per_s": float(qs.lengths()[pr["status"] == 0].sum()) / t_pr / 1e9,
                       "cells": int(pr["cells"].sum()), "upper_bound_rate": float(pr["is_upper_bound"].mean()),
                       "ok": int((pr["status"] == 0).sum())},
            "exact": {"queries": n_exact, "s": t_ex,
                      "gbp_per_s": float(sub.lengths()[ex["status"] == 0].sum()) / t_ex / 1e9,
                      "cells": int(ex["cells"].sum()), "ok": int((ex["status"] == 0).sum()),
                      "mean_distance": float(ex["edit_distance"][ex["status"] == 0].mean())},
            "bounded_memory": dict(bounded, unbounded_engine_bytes=free_bytes,
                                   unbounded_tier0_overflows=free_retries,
                                   exact_match_rate=float((bd["edit_distance"][:n_exact][ok] ==
                                                           ex["edit_distance"][ok]).mean())),
            "exact_match_rate": float((prs["edit_distance"][ok] == ex["edit_distance"][ok]).mean()),
            "pruned_never_below_exact": bool(np.all(prs["edit_distance"][ok] >= ex["edit_distance"][ok])),
            "work_ratio_exact_over_pruned": float(ex["cells"][ok].sum() / max(prs["cells"][ok].sum(), 1))}


def _trained_model(n_train_c2: int = 3000, n_train_c3: int = 300):
    """Cost model trained on wave logs of config-2 queries and of queries on the
    config-3 graph (graphs other than the large one it is used on); also the fitted
    per-score / per-cell time coefficients."""
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import costmodel, synth
    import torch
    # training logs on the two other graphs
    g2, q2 = synth.make_config(2, n_queries=n_train_c2, seed=12)
    c3 = synth.CONFIGS[3]
    g3 = synth.make_graph(c3["graph"], 3)
    q3 = synth.make_queries(g3, n_train_c3, 13, lambda r: r.one_int(3000, 15000), lambda r: 0.005 + 0.05 * r.one(),
                            c3["weights"], c3["loops"])
    feats, tgts = [], []
    gr2 = gw.Graph.from_synth(g2)
    m2 = gw.CostModel(gr2, seed=1)
    f, t, r2res = costmodel.collect(m2, gw.Engine(gr2), q2)
    feats.append(f)
    tgts.append(t)
    coeffs = costmodel.time_coeffs(r2res)
    gr3 = gw.Graph.from_synth(g3)
    m3 = gw.CostModel(gr3, seed=1)
    cfg3 = gw.default_config(gr3)
    cfg3.tiers[1].log2_tiles, cfg3.tiers[2].log2_tiles = 20, 23
    f, t, _ = costmodel.collect(m3, gw.Engine(gr3, config=cfg3), q3)
    feats.append(f)
    tgts.append(t)
    feat = torch.cat(feats)
    tgt = torch.cat(tgts)
    costmodel.fit(m2, feat, tgt, steps=2000, batch=512, lr=3e-3)
    return m2, coeffs


def scheduler(n: int = 5000, n_train_c2: int = 3000, n_train_c3: int = 300, n_plain: int = 100,
              only=None) -> dict:
    """Large graph (50 Mb, lognormal 1-100 kb queries, 0.1-10% divergence), exact:
    plain schedules (input order, longest first) against the learned plan of a cost
    model trained on config-2 and config-3-graph logs (other graphs)."""
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import costmodel, synth
    m2, coeffs = _trained_model(n_train_c2, n_train_c3)
    # the large workload
    g4, q4 = synth.make_config(4, n_queries=n)
    gr4 = gw.Graph.from_synth(g4)
    m4 = gw.CostModel(gr4, seed=1)
    costmodel.transfer(m2, m4)
    b0 = gw.DeviceBatch(q4)
    pred = m4.predict(m4.features(b0)).cpu().numpy()
    base = gw.default_config(gr4)
    total = base.tiers[0].ctas
    wide_log2, huge_log2 = 20, 23

    def engine(wide: int = 0, huge: int = 0, huge_threads: int = 1024):
        cfg = gw.default_config(gr4)
        cfg.tiers[1].ctas, cfg.tiers[1].log2_tiles = 152, 20
        cfg.tiers[2].ctas, cfg.tiers[2].log2_tiles = 19, 23
        cfg.wide.ctas, cfg.wide.log2_tiles, cfg.wide.threads = wide, wide_log2, 512
        cfg.huge.ctas, cfg.huge.log2_tiles, cfg.huge.threads = huge, huge_log2, huge_threads
        return gw.Engine(gr4, config=cfg)

    probe = engine(1, 1).config
    l_order, l_huge, l_wide = gw.plan_schedule(pred, *costmodel.capacities(probe))
    # one CTA per huge query (they are few and each is a long tail on its own);
    # wide CTAs by the wide class's share of the predicted time
    h_ctas = min(l_huge, 32)
    w_ctas = costmodel.wide_ctas(pred, l_order, l_wide, total, coeffs, first=l_huge)
    out = {"workload": f"config4: 50 Mb graph, {n} lognormal 1-100 kb queries, 0.1-10% divergence, exact",
           "train": f"{n_train_c2} config-2 + {n_train_c3} config-3-graph queries, 2000 Adam steps",
           "learned_huge": [int(l_huge), int(h_ctas), huge_log2], "learned_wide": [int(l_wide), int(w_ctas), wide_log2],
           "time_coeffs_us": list(coeffs)}
    ref = None
    # (order, n_huge, n_wide, huge CTAs, wide CTAs, threads per huge CTA)
    plans = {"plain_fifo": (None, 0, 0, 0, 0, 512),
             "plain_longest_first": (np.argsort(-q4.lengths(), kind="stable"), 0, 0, 0, 0, 512)}
    o2, _, nw2 = gw.plan_schedule(pred, int(0.75 * (1 << base.tiers[0].log2_tiles)))
    plans["learned_wide_only"] = (o2, 0, nw2, 0, costmodel.wide_ctas(pred, o2, nw2, total, coeffs), 512)
    plans["learned_huge_512_threads"] = (l_order, l_huge, l_wide, h_ctas, w_ctas, 512)
    plans["learned"] = (l_order, l_huge, l_wide, h_ctas, w_ctas, 1024)
    if only is not None:
        plans = {k: v for k, v in plans.items() if k in only}
    for name, (order, nh, nw, hc, wc, hth) in plans.items():
        eng = engine(wc, hc, hth)
        b = gw.DeviceBatch(q4, order=None if order is None else np.asarray(order, np.uint32))
        b.run(eng, n_wide=nw, n_huge=nh)
        t = _timed_run(eng, b, n_wide=nw, n_huge=nh)
        r = b.results()
        retries = eng.last_retries()
        if ref is None:
            ref = r
        assert np.array_equal(r["edit_distance"], ref["edit_distance"])
        out[name] = {"s": t, "gbp_per_s": float(q4.lengths()[r["status"] == 0].sum()) / t / 1e9,
                     "tier0_overflows": int(retries[0]), "tier1_overflows": int(retries[1]),
                     "n_huge": int(nh), "n_wide": int(nw), "huge_ctas": int(hc), "wide_ctas": int(wc),
                     "huge_threads": int(hth), "ok": int((r["status"] == 0).sum()),
                     "slab_bytes": eng.device_bytes, "slowest_query_ms": float(r["device_us"].max() / 1e3)}
        eng.close()
    # where the time goes: the heaviest queries' own CTA times against the batch
    top = np.argsort(-ref["device_us"].astype(np.float64))[:8]
    out["slowest_queries"] = [{"len": int(q4.lengths()[i]), "us": int(ref["device_us"][i]),
                               "cells": int(ref["cells"][i]), "visited": int(ref["visited"][i])} for i in top]
    # S4 on the same workload: the plain path, one synchronous launch per query
    if n_plain:
        rng = np.random.default_rng(4)
        sidx = rng.choice(len(q4), size=min(n_plain, len(q4)), replace=False)
        t0 = time.perf_counter()
        for i in sidx:
            r = gr4.align(q4.query(int(i)), int(q4.v_s[i]), int(q4.v_e[i]))
            assert r["edit_distance"] == int(ref["edit_distance"][i])
        tp = time.perf_counter() - t0
        out["plain_per_query"] = {"queries": int(len(sidx)), "s": tp,
                                  "gbp_per_s": float(q4.lengths()[sidx].sum()) / tp / 1e9,
                                  "ms_per_query": tp / len(sidx) * 1e3}
    out["cells"] = int(ref["cells"].sum())
    out["spearman_pred_cells"] = costmodel.spearman(pred[:, 3], np.log1p(ref["cells"].astype(np.float64)))
    out["r2_log_cells"] = float(costmodel.r2(pred[:, 3:4], np.log1p(ref["cells"].astype(np.float64))[:, None])[0])
    return out


def serving(n_pool: int = 3000, rates=(1000.0, 5000.0, 20000.0), duration: float = 1.0,
            plain_rate: float = 100.0, plain_duration: float = 2.0, cfg: int = 2,
            with_model: bool = False) -> dict:
    """A resident graph, Poisson arrivals: the continuous-batching server's p50/p99 at
    several rates, and the plain one-query-at-a-time path at a low rate.  cfg 2: the
    config-2 graph and queries; cfg 5: the 50 Mb config-4 graph with its lognormal
    1-100 kb queries at 0.1-10% divergence."""
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import serving as sv
    from paper_2206_13574_gb300 import synth
    g, qs = synth.make_config(cfg, n_queries=n_pool)
    graph = gw.Graph.from_synth(g)
    srv = gw.Server(graph)
    out = {"workload": ("config2 graph, config-2 queries" if cfg == 2 else
                        "config5: 50 Mb config-4 graph resident, lognormal 1-100 kb queries, 0.1-10% divergence")
                       + ", Poisson arrivals"}
    for lam in rates:
        arr = synth.poisson_arrivals(lam, duration, seed=int(lam))
        idx = np.arange(len(arr)) % n_pool
        out[f"server_lambda_{int(lam)}"], _ = sv.run_server(srv, qs, arr, idx)
    out["server_stats"] = srv.stats()
    srv.close()
    if with_model:
        # admission by the cost model's predicted memory instead of the query length
        from paper_2206_13574_gb300 import costmodel
        m_src, _ = _trained_model()
        model = gw.CostModel(graph, seed=1)
        costmodel.transfer(m_src, model)
        srvm = gw.Server(graph, model=model)
        for lam in rates:
            arr = synth.poisson_arrivals(lam, duration, seed=int(lam))
            idx = np.arange(len(arr)) % n_pool
            out[f"model_server_lambda_{int(lam)}"], _ = sv.run_server(srvm, qs, arr, idx)
        out["model_server_stats"] = srvm.stats()
        srvm.close()
    arr = synth.poisson_arrivals(plain_rate, plain_duration, seed=3)
    idx = np.arange(len(arr)) % n_pool
    out[f"plain_lambda_{int(plain_rate)}"], _ = sv.run_plain(graph, qs, arr, idx)
    srv2 = gw.Server(graph)
    out[f"server_lambda_{int(plain_rate)}"], _ = sv.run_server(srv2, qs, arr, idx)
    srv2.close()
    return out


if __name__ == "__main__":
    import paper_2206_13574_gb300._build as b
    b.build()
    which = sys.argv[1] if len(sys.argv) > 1 else "config3"
    t0 = time.time()
    res = {"config3": config3, "scheduler": scheduler, "serving": serving,
           "scheduler100k": lambda: scheduler(n=100_000, n_plain=0, only=("plain_fifo", "learned")),
           "serving5": lambda: serving(n_pool=3000, rates=(1000.0, 2000.0, 5000.0, 10000.0), duration=4.0,
                                       plain_rate=10.0, plain_duration=3.0, cfg=5, with_model=True)}[which]()
    res["wall_s"] = time.time() - t0
    print(json.dumps(res))

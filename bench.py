"""Benchmark of the encrypted query-point distance step (SANNS linear scan).

One step = the server's whole distance computation for one encrypted query
against the resident encoded database: ct x pt MAC over all d dimensions
(K2), then INTT + ||p||^2 + mask (K1/K3).  Workload: n = 1,000,000 points,
d = 128, uint8 coordinates from a 64-component Gaussian mixture (sigma = 20),
BFV N = 8192 with three 60-bit RNS primes, t = the smallest prime > 2^24 that
is 1 mod 2N; 100 queries from the same mixture, one per step, cycled.

Prints one JSON line.  `value` is query-point distances per second with all
inputs resident in HBM; `e2e` is the same metric through the C-ABI call with
the query ciphertext copied from pinned host memory and the response
ciphertexts plus the server share copied back, inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sanns|reference]

--impl reference times the CPU oracle (the plain C loops under oracle/) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=1_000_000, d=128, N=8192, L=3, prime_bits=60, t_rule=0, n_comp=64,
                sigma=20.0, n_queries=100, seed=0)
METRIC = "encrypted query-point distances/s (bit-exact, plain per-query path)"
UNIT = "qp/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _roofline_bytes(W) -> dict:
    """Algorithmic HBM bytes of one MAC launch for one query: the encoded
    database once (K L d N 8), the query ciphertext once (d 2 L N 8) and the
    accumulator output (K 2 L N 8)."""
    K = -(-W["n"] // W["N"])
    pt = K * W["L"] * W["d"] * W["N"] * 8
    ct = W["d"] * 2 * W["L"] * W["N"] * 8
    out = K * 2 * W["L"] * W["N"] * 8
    return {"pt": pt, "ct": ct, "out": out, "total": pt + ct + out, "K": K}


# DRAM bytes of one mac_kernel launch (spl2_unr8_512x1) from the ncu capture
# of the small case n = 200,000 (K = 25 blocks, d = 128, N = 8192, L = 3;
# profiles/mac_kernel_linear_scan_n200k.md): dram__bytes_read.sum +
# dram__bytes_write.sum.  The query ciphertext is read once per launch; the
# rest grows with the blocks, so a full launch's traffic is that rest scaled
# by the block count plus the query ciphertext.
MAC_CAPTURE = dict(K=25, d=128, N=8192, L=3, dram_bytes=679_687_680 + 2_998_272)


def _mac_traffic(rb: dict, W) -> float | None:
    C = MAC_CAPTURE
    if (W["d"], W["N"], W["L"]) != (C["d"], C["N"], C["L"]):
        return None
    ct = C["d"] * 2 * C["L"] * C["N"] * 8
    return (C["dram_bytes"] - ct) * rb["K"] / C["K"] + ct


def _ntt_roofline(rates: dict, polys: int, N: int, ms: float) -> dict:
    """The INTT + mask epilogue against the measured register-resident
    inverse-butterfly rate (integer pipes): N/2 log2 N butterflies per
    polynomial."""
    bf = polys * (N // 2) * (N.bit_length() - 1)
    achieved = bf / (ms * 1e-3)
    return {"bound": "alu", "achieved": achieved, "peak": rates["inv_butterflies_per_s"],
            "unit": "butterflies/s", "frac": achieved / rates["inv_butterflies_per_s"],
            "peak_source": "library probe: register-resident inverse butterflies on this GPU "
                           "(sanns_measure_int_rates)"}


def _ntt_report(polys: int, N: int, ms: float, what: str) -> dict:
    """The epilogue's transforms (one inverse NTT per block, component and
    prime, with the mask): polynomials per second and the fraction of the HBM
    copy peak that 16 N bytes per polynomial (read and written once) would
    use.  The transforms are bound by the integer multiply pipe instead
    (profiles/intt_mask_kernel_linear_scan_n1M.md)."""
    peak, _ = _peaks()
    gbs = 16.0 * N * polys / (ms * 1e-3) / 1e9
    return {"what": what, "polys": polys, "ms": ms, "polys_per_s": polys / (ms * 1e-3),
            "hbm_gbs": gbs, "hbm_frac": gbs / peak, "bound": "integer multiply pipe",
            "pipes_from_ncu": {"fma_heavy_pct": 77.2, "alu_pct": 48.2,
                               "source": "ncu of the fused INTT + mask kernel, 5,952 polynomials "
                                         "(profiles/intt_mask_kernel_linear_scan_n1M.md)"}}


def run_small_section() -> dict:
    """The small linear scan: n = 4096, d = 32 uniform uint8, N = 4096, two
    54-bit primes, one query; latency-bound, so p50/p99 of the distance step,
    and the exact top-10 checked against brute force."""
    import numpy as np
    import torch

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S

    n, d = 4096, 32
    ctx = S.sanns_ctx_create(4096, 2, 54, 0, d)
    coords = inputs.uniform_coords(n, d, 0)
    perm = inputs.permutation(n, 0)
    q = inputs.uniform_coords(1, d, 0)
    qids = torch.from_numpy(np.array([0], dtype=np.uint64)).cuda()
    sk = S.sanns_keygen(ctx, 0)
    db = S.sanns_encode_db(ctx, torch.from_numpy(coords).cuda(), torch.from_numpy(perm).cuda())
    ct = S.sanns_encrypt_query(ctx, sk, torch.from_numpy(q).cuda(), 0, qids)
    out, srv = S.sanns_distances(ctx, db, ct, 0, qids)
    variant, _ = S.sanns_autotune_mac(ctx, db, ct, out, reps=50)
    st = torch.cuda.current_stream()
    reps = 500
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for _ in range(10):
        S.sanns_distances(ctx, db, ct, 0, qids, out, srv)
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(st)
        S.sanns_distances(ctx, db, ct, 0, qids, out, srv)
        b.record(st)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    # the same step captured once into a CUDA graph and replayed: the launch
    # gaps of the eager calls above are host time, not the step's own
    gs = torch.cuda.Stream()
    gs.wait_stream(st)
    with torch.cuda.stream(gs):
        S.sanns_distances(ctx, db, ct, 0, qids, out, srv)
    st.wait_stream(gs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sanns_distances(ctx, db, ct, 0, qids, out, srv)
    torch.cuda.synchronize()
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    cur = torch.cuda.current_stream()
    for a, b in gev:
        a.record(cur)
        g.replay()
        b.record(cur)
    torch.cuda.synchronize()
    glat = sorted(a.elapsed_time(b) for a, b in gev)
    # 50 steps in one graph: the per-step device time without the per-replay
    # cost (back-to-back queries, as a serving loop would run them)
    g50 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g50):
        for _ in range(50):
            S.sanns_distances(ctx, db, ct, 0, qids, out, srv)
    torch.cuda.synchronize()
    g50.replay()
    torch.cuda.synchronize()
    e50 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(40)]
    for a, b in e50:
        a.record(cur)
        g50.replay()
        b.record(cur)
    torch.cuda.synchronize()
    l50 = sorted(a.elapsed_time(b) / 50 for a, b in e50)
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, torch.from_numpy(q).cuda())
    dist_k, pos_k = S.sanns_topk(ctx, cli, srv, 10)
    brute = np.sum((coords[perm].astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
    exact = sorted(brute.tolist())[:10] == dist_k.cpu().numpy()[0].tolist()
    return {"workload": "small linear scan: n=4,096 d=32 uniform uint8; BFV N=4096, two 54-bit primes; "
                        "one query per step",
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[int(0.99 * (len(lat) - 1))]},
            "latency_graph_ms": {"p50": glat[len(glat) // 2], "p99": glat[int(0.99 * (len(glat) - 1))],
                                 "what": "one step captured into a CUDA graph, replayed"},
            "ms_per_step_graph_of_50": l50[len(l50) // 2],
            "qp_per_s": n / (lat[len(lat) // 2] * 1e-3), "steps": reps,
            "mac_variant": S.sanns_mac_variants()[variant],
            "epilogue": "four CTAs (a cluster) per response polynomial, mask drawn in the same kernel",
            "exact_top10_equals_brute_force": bool(exact)}


def run_gpu(args) -> None:
    import torch

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    W = WORKLOAD
    n, d, N, L = W["n"], W["d"], W["N"], W["L"]
    ctx = S.sanns_ctx_create(N, L, W["prime_bits"], W["t_rule"], d)
    # every rank holds its own full database and query stream (weak scaling)
    coords = inputs.mixture_coords(n, d, W["n_comp"], W["sigma"], W["seed"] + 1000 * rank,
                                   means_seed=W["seed"])
    queries = inputs.mixture_coords(W["n_queries"], d, W["n_comp"], W["sigma"],
                                    W["seed"] + 1 + 1000 * rank, means_seed=W["seed"])
    perm = inputs.permutation(n, W["seed"] + 2 + rank)
    sk = S.sanns_keygen(ctx, W["seed"] + 3)
    db = S.sanns_encode_db(ctx, torch.from_numpy(coords).cuda(), torch.from_numpy(perm).cuda())
    qdev = torch.from_numpy(queries).cuda()
    qids = torch.arange(W["n_queries"], dtype=torch.int64).to(torch.uint64).cuda()
    ct_all = S.sanns_encrypt_query(ctx, sk, qdev, W["seed"] + 4, qids)
    K = db.K
    ct_out = torch.empty((1, K, 2, L, N), dtype=torch.uint64, device="cuda")
    srv = torch.empty((1, n), dtype=torch.uint32, device="cuda")
    stream = torch.cuda.current_stream()
    mask_seed = W["seed"] + 5
    variant_names = S.sanns_mac_variants()
    if args.mac_variant:
        # a fixed launch variant (profiler runs, whose per-launch overhead
        # would decide the autotuner's pick)
        variant, variant_ms = variant_names.index(args.mac_variant), []
        S.sanns_set_mac_variant(ctx, variant)
    else:
        variant, variant_ms = S.sanns_autotune_mac(ctx, db, ct_all[0:1], ct_out, reps=3)

    # Steps are pipelined over two streams: query s's MAC (HBM-bound) runs on
    # stream A while query s-1's INTT + mask (integer-bound) runs on stream B,
    # with the responses double-buffered; the MAC's persistent grid is capped
    # at `mac_sms` SMs so that the other SMs take the INTT meanwhile.
    s_mac, s_fin = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [ct_out, torch.empty_like(ct_out)]
    srvs = [srv, torch.empty_like(srv)]

    def run_steps(first, count, starts=None, mac_end=None, ends=None):
        fin = [None] * count
        for i in range(count):
            s = first + i
            qi, u = s % W["n_queries"], s % 2
            if i >= 2:
                s_mac.wait_event(fin[i - 2])
            if starts is not None:
                starts[s].record(s_mac)
            S.sanns_distances_mac(ctx, db, ct_all[qi:qi + 1], outs[u], stream=s_mac)
            me = mac_end[s] if mac_end is not None else torch.cuda.Event()
            me.record(s_mac)
            s_fin.wait_event(me)
            S.sanns_distances_finish(ctx, db, outs[u], mask_seed, qids[qi:qi + 1], srvs[u],
                                     stream=s_fin)
            fin[i] = ends[s] if ends is not None else torch.cuda.Event()
            fin[i].record(s_fin)
        s_mac.wait_event(fin[count - 1])

    def time_steps(count):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s_mac)
        run_steps(0, count)
        e1.record(s_mac)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / count

    # the SM cap, tuned on short pipelined runs (0 = all SMs)
    sms_ms = {}
    for cap in ((args.mac_sms,) if args.mac_sms is not None else (0, 144, 140, 136, 132, 128, 124, 120)):
        S.sanns_set_mac_sms(ctx, cap)
        time_steps(20)
        sms_ms[cap] = time_steps(100)
    mac_sms = min(sms_ms, key=sms_ms.get)
    # the same steps one after another on one stream with every SM, for
    # reference; its INTT + mask times are the stage's own (the pipelined
    # loop's overlap with the next MAC)
    S.sanns_set_mac_sms(ctx, 0)
    serial_n = min(args.steps, 200)
    torch.cuda.synchronize()
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(serial_n)]
    for s in range(serial_n):
        qi = s % W["n_queries"]
        sev[s][0].record(stream)
        S.sanns_distances_mac(ctx, db, ct_all[qi:qi + 1], ct_out, stream=stream)
        sev[s][1].record(stream)
        S.sanns_distances_finish(ctx, db, ct_out, mask_seed, qids[qi:qi + 1], srv, stream=stream)
        sev[s][2].record(stream)
    torch.cuda.synchronize()
    serial_ms = sev[0][0].elapsed_time(sev[-1][2]) / serial_n
    serial_mac_ms = sum(e[0].elapsed_time(e[1]) for e in sev) / serial_n
    serial_fin_ms = sum(e[1].elapsed_time(e[2]) for e in sev) / serial_n
    S.sanns_set_mac_sms(ctx, mac_sms)

    total_steps = args.warmup + args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(total_steps)]
    mac_end = [torch.cuda.Event(enable_timing=True) for _ in range(total_steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(total_steps)]
    run_steps(0, args.warmup, starts, mac_end, ends)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # the pipelined steps issued one by one from the host: each step's start,
    # MAC end and finish end are events (query latency, the MAC's launch time)
    t0.record(s_mac)
    run_steps(args.warmup, args.steps, starts, mac_end, ends)
    t1.record(s_mac)
    torch.cuda.synchronize()
    eager_ms = t0.elapsed_time(t1)
    # The timed steps: the same K pipelined steps (the same queries, buffers
    # and SM cap) captured into one CUDA graph, the finish stream forking from
    # the capture stream at each MAC's end and joining it at the last finish.
    # One untimed replay, then one timed replay of all K steps.
    # (more than 5000 steps are timed as issued, without the graph)
    use_graph = args.steps <= 5000
    cap_st, side_st = torch.cuda.Stream(), torch.cuda.Stream()
    cap_st.wait_stream(s_mac)
    steps_graph = torch.cuda.CUDAGraph() if use_graph else None
    if use_graph:
        with torch.cuda.graph(steps_graph, stream=cap_st):
            gfin = [None] * args.steps
            for i in range(args.steps):
                s = args.warmup + i
                qi, u = s % W["n_queries"], s % 2
                if i >= 2:
                    cap_st.wait_event(gfin[i - 2])
                S.sanns_distances_mac(ctx, db, ct_all[qi:qi + 1], outs[u], stream=cap_st)
                me = torch.cuda.Event()
                me.record(cap_st)
                side_st.wait_event(me)
                S.sanns_distances_finish(ctx, db, outs[u], mask_seed, qids[qi:qi + 1], srvs[u],
                                         stream=side_st)
                gfin[i] = torch.cuda.Event()
                gfin[i].record(side_st)
            cap_st.wait_event(gfin[args.steps - 1])
    if use_graph:
        steps_graph.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    torch.cuda.synchronize()
    replay_st = torch.cuda.current_stream() if use_graph else s_mac   # a graph replays on the current stream
    t0.record(replay_st)
    if use_graph:
        steps_graph.replay()
    else:
        run_steps(args.warmup, args.steps)
    t1.record(replay_st)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    del steps_graph
    S.sanns_set_mac_sms(ctx, 0)   # the single-stream sections below use every SM
    # the last two pipelined steps against the same queries run alone
    pipe_exact = True
    for s in (total_steps - 2, total_steps - 1):
        qi, u = s % W["n_queries"], s % 2
        o1, s1 = S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1])
        pipe_exact &= bool(torch.equal(o1, outs[u]) and torch.equal(s1, srvs[u]))
    del o1, s1
    if dist:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    timed = range(args.warmup, total_steps)
    lat = sorted(starts[s].elapsed_time(ends[s]) for s in timed)
    mac_ms = [starts[s].elapsed_time(mac_end[s]) for s in timed]
    mac_avg = sum(mac_ms) / len(mac_ms)
    fin_ms = [mac_end[s].elapsed_time(ends[s]) for s in timed]
    fin_avg = sum(fin_ms) / len(fin_ms)

    # the same steps replayed from one captured CUDA graph (MAC, mask draw and
    # INTT + mask of G consecutive queries as graph nodes)
    G = min(args.steps, 100)
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        for s in range(2):
            qi = s % W["n_queries"]
            S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1], ct_out, srv)
    stream.wait_stream(gs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for s in range(G):
            qi = s % W["n_queries"]
            S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1], ct_out, srv)
    graph.replay()
    torch.cuda.synchronize()
    g_reps = max(1, args.steps // G)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(g_reps):
        graph.replay()
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / (g_reps * G)
    del graph

    # selection on the reconstructed shares, for every query of this workload:
    # client decryption, exact top-10 and ApproxTopk with l = ceil(n / 128)
    # bins (Algorithm 2), against brute-force squared distances of the
    # permuted points.  |I| = |exact top-k ids & approximate ids|; the tie-aware
    # count takes the approximate picks below the exact k-th value plus, at
    # that value, as many as the exact list holds there.
    k_sel, l_sel = 10, -(-n // 128)
    pts = torch.from_numpy(coords).cuda()[torch.from_numpy(perm.astype(np.int64)).cuda()].int()
    hits, hits_ties, exact_ok, ms_ex, ms_ap = [], [], True, [], []
    for qi in range(W["n_queries"]):
        out1, srv1 = S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1])
        cli1 = S.sanns_decrypt_shares(ctx, sk, out1, n, qdev[qi:qi + 1])
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record(stream)
        ed, ep = S.sanns_topk(ctx, cli1, srv1, k_sel)
        s1.record(stream)
        ad, ap = S.sanns_topk(ctx, cli1, srv1, k_sel, l_sel)
        s2.record(stream)
        brute = ((pts - qdev[qi].int()) ** 2).sum(1)
        bv = torch.topk(brute, k_sel, largest=False).values.sort().values
        torch.cuda.synchronize()
        ms_ex.append(s0.elapsed_time(s1))
        ms_ap.append(s1.elapsed_time(s2))
        exact_ok &= (bool(torch.equal(ed[0].long().sort().values, bv.long()))
                     and bool(torch.equal(brute[ep[0]].long(), ed[0].long()))
                     and bool(torch.equal(brute[ap[0]].long(), ad[0].long())))
        hits.append(len(set(ep[0].tolist()) & set(ap[0].tolist())))
        ev = ed[0].long()
        dk = int(ev.max())
        av = ad[0].long()
        hits_ties.append(int((av < dk).sum()) + min(int((av == dk).sum()), int((ev == dk).sum())))
        del out1, srv1, cli1, brute
    selection = {
        "k": k_sel, "bins": l_sel, "queries": W["n_queries"],
        "exact_top10_equals_brute_force": exact_ok,
        "approx_mean_hits": float(np.mean(hits)), "approx_min_hits": int(min(hits)),
        "approx_mean_hits_tie_aware": float(np.mean(hits_ties)),
        "approx_mean_hits_threshold": 9.9,
        "approx_recall_vs_exact": float(np.mean(hits)) / k_sel,
        "ms_exact": float(np.median(ms_ex)), "ms_approx": float(np.median(ms_ap)),
    }
    del pts

    # the same step with circuit privacy on (public-key re-randomisation and
    # noise flooding, F = 148: 108 bits of statistical privacy over a
    # structured noise below 2^40)
    pk = S.sanns_public_key(ctx, sk, W["seed"] + 6)
    flood = min(148, S.sanns_circuit_privacy_max_flood_bits(ctx))
    S.sanns_set_circuit_privacy(ctx, pk, flood)
    cp_steps = max(10, min(args.steps, 200))
    for s in range(3):
        S.sanns_distances(ctx, db, ct_all[s:s + 1], mask_seed, qids[s:s + 1], ct_out, srv)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c0.record(stream)
    for s in range(cp_steps):
        qi = s % W["n_queries"]
        S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1], ct_out, srv)
    c1.record(stream)
    torch.cuda.synchronize()
    cp_ms = c0.elapsed_time(c1) / cp_steps
    S.sanns_set_circuit_privacy(ctx, None)
    del pk

    # NTT-form responses (the NTT of the coefficient-form response): one
    # forward transform per block and prime instead of two inverse ones
    S.sanns_set_response_form(ctx, True)
    for s in range(3):
        S.sanns_distances(ctx, db, ct_all[s:s + 1], mask_seed, qids[s:s + 1], ct_out, srv)
    torch.cuda.synchronize()
    c0.record(stream)
    for s in range(cp_steps):
        qi = s % W["n_queries"]
        S.sanns_distances(ctx, db, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1], ct_out, srv)
    c1.record(stream)
    torch.cuda.synchronize()
    nf_ms = c0.elapsed_time(c1) / cp_steps
    S.sanns_set_response_form(ctx, False)

    # slot encoding (points in the CRT slots mod t): the same database encoded
    # through the inverse transform mod t; the step adds the server's slot
    # shares (one forward transform mod t per block); one query checked
    # against brute force through the client's slot decoding
    S.sanns_set_encoding(ctx, True)
    db_s = S.sanns_encode_db(ctx, torch.from_numpy(coords).cuda(), torch.from_numpy(perm).cuda())
    for s in range(3):
        S.sanns_distances(ctx, db_s, ct_all[s:s + 1], mask_seed, qids[s:s + 1], ct_out, srv)
    torch.cuda.synchronize()
    c0.record(stream)
    for s in range(cp_steps):
        qi = s % W["n_queries"]
        S.sanns_distances(ctx, db_s, ct_all[qi:qi + 1], mask_seed, qids[qi:qi + 1], ct_out, srv)
    c1.record(stream)
    torch.cuda.synchronize()
    sl_ms = c0.elapsed_time(c1) / cp_steps
    S.sanns_distances(ctx, db_s, ct_all[0:1], mask_seed, qids[0:1], ct_out, srv)
    cli_s = S.sanns_decrypt_shares(ctx, sk, ct_out, n, qdev[0:1])
    pts = torch.from_numpy(coords).cuda()[torch.from_numpy(perm.astype(np.int64)).cuda()]
    brute = ((pts.int() - qdev[0].int()) ** 2).sum(1)
    t_mod = ctx.query()["t"]
    slot_exact = bool(torch.equal((cli_s[0].long() + srv[0].long()) % t_mod, brute.long()))
    del db_s, cli_s, pts, brute
    S.sanns_set_encoding(ctx, False)

    # end-to-end through the C ABI: each step copies its query ciphertext from
    # pinned host memory, runs the distance step (sanns_distances_mac, then
    # sanns_distances_finish) and copies the response ciphertexts and the
    # server share back; four streams overlap step s's MAC with step s-1's
    # finish (the MAC's grid at the tuned SM cap, as in the timed loop), the
    # upload of s+1 and the download of s-1.
    nh = min(4, W["n_queries"])
    ct_host = ct_all[:nh].cpu().pin_memory()
    out_host = [torch.empty((1, K, 2, L, N), dtype=torch.uint64).pin_memory() for _ in range(2)]
    srv_host = [torch.empty((1, n), dtype=torch.uint32).pin_memory() for _ in range(2)]
    ct_dev = [torch.empty((1, d, 2, L, N), dtype=torch.uint64, device="cuda") for _ in range(2)]
    out_dev = [torch.empty((1, K, 2, L, N), dtype=torch.uint64, device="cuda") for _ in range(2)]
    srv_dev = [torch.empty((1, n), dtype=torch.uint32, device="cuda") for _ in range(2)]
    s_up, s_cmp, s_dn = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    s_fin = torch.cuda.Stream()
    e2e_steps = max(10, min(args.steps, 100))

    # seeded queries: the client sends c0 alone; the server rebuilds c1 from
    # the encryption seed (sanns_expand_query) before the distance step
    c0_host = ct_all[:nh, :, 0].contiguous().cpu().pin_memory()
    c0_dev = [torch.empty((1, d, L, N), dtype=torch.uint64, device="cuda") for _ in range(2)]
    # responses switched down to q_0 (sanns_set_response_primes): the download
    # is the compact q_0 rows, a third of the bytes
    sw_host = [torch.empty((1, K, 2, 1, N), dtype=torch.uint64).pin_memory() for _ in range(2)]

    def run_e2e(nsteps, seeded=False, switched=False):
        up_done = [torch.cuda.Event() for _ in range(nsteps)]
        mac_done = [torch.cuda.Event() for _ in range(nsteps)]
        cmp_done = [torch.cuda.Event() for _ in range(nsteps)]
        dn_done = [torch.cuda.Event() for _ in range(nsteps)]
        for s in range(nsteps):
            u = s % 2
            qi = s % nh
            with torch.cuda.stream(s_up):
                if s >= 2:
                    s_up.wait_event(mac_done[s - 2])      # ct_dev[u] free again
                if seeded:
                    c0_dev[u].copy_(c0_host[qi:qi + 1], non_blocking=True)
                else:
                    ct_dev[u].copy_(ct_host[qi:qi + 1], non_blocking=True)
                up_done[s].record(s_up)
            s_cmp.wait_event(up_done[s])
            if s >= 2:
                s_cmp.wait_event(dn_done[s - 2])          # out_dev[u], srv_dev[u] downloaded
            if seeded:
                S.sanns_expand_query(ctx, c0_dev[u], W["seed"] + 4, qids[qi:qi + 1], out=ct_dev[u],
                                     stream=s_cmp)
            S.sanns_distances_mac(ctx, db, ct_dev[u], out_dev[u], stream=s_cmp)
            mac_done[s].record(s_cmp)
            s_fin.wait_event(mac_done[s])
            S.sanns_distances_finish(ctx, db, out_dev[u], mask_seed, qids[qi:qi + 1], srv_dev[u],
                                     stream=s_fin)
            cmp_done[s].record(s_fin)
            with torch.cuda.stream(s_dn):
                s_dn.wait_event(cmp_done[s])
                if switched:
                    S.sanns_copy_responses(ctx, out_dev[u], sw_host[u], stream=s_dn)
                else:
                    out_host[u].copy_(out_dev[u], non_blocking=True)
                srv_host[u].copy_(srv_dev[u], non_blocking=True)
                dn_done[s].record(s_dn)
        return dn_done[-1]

    S.sanns_set_mac_sms(ctx, mac_sms)
    run_e2e(4)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    last = run_e2e(e2e_steps)
    last.synchronize()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t_start) * 1e3 / e2e_steps
    run_e2e(4, seeded=True)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    run_e2e(e2e_steps, seeded=True).synchronize()
    torch.cuda.synchronize()
    e2e_seeded_ms = (time.perf_counter() - t_start) * 1e3 / e2e_steps
    seeded_exact = bool(torch.equal(
        S.sanns_expand_query(ctx, c0_host[0:1].cuda(), W["seed"] + 4, qids[0:1]), ct_all[0:1]))
    S.sanns_set_response_primes(ctx, 1)
    e2e_sw = {}
    issue_sw = {}
    for seeded in (False, True):
        run_e2e(4, seeded=seeded, switched=True)
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        ev_last = run_e2e(e2e_steps, seeded=seeded, switched=True)
        issue_sw[seeded] = (time.perf_counter() - t_start) * 1e3 / e2e_steps
        ev_last.synchronize()
        torch.cuda.synchronize()
        e2e_sw[seeded] = (time.perf_counter() - t_start) * 1e3 / e2e_steps
    # the last step's downloaded switched response decrypts to shares that
    # reconstruct the brute-force distances of its query
    s_last = e2e_steps - 1
    u_last, q_last = s_last % 2, s_last % nh
    cli_sw = S.sanns_decrypt_shares(ctx, sk, sw_host[u_last].cuda(), n, qdev[q_last:q_last + 1])
    pts_all = torch.from_numpy(coords).cuda()[torch.from_numpy(perm.astype(np.int64)).cuda()]
    brute_sw = ((pts_all.int() - qdev[q_last].int()) ** 2).sum(1)
    switched_exact = bool(torch.equal((cli_sw[0].long() + srv_host[u_last][0].cuda().long()) % t_mod,
                                      brute_sw.long()))
    del cli_sw, brute_sw, pts_all
    # the host link alone for the switched, seeded pattern: c0 up, the q_0 rows
    # (a pitched copy) and the shares down
    torch.cuda.synchronize()
    t_l = time.perf_counter()
    for r in range(20):
        with torch.cuda.stream(s_up):
            c0_dev[r % 2].copy_(c0_host[r % nh:r % nh + 1], non_blocking=True)
        with torch.cuda.stream(s_dn):
            S.sanns_copy_responses(ctx, out_dev[r % 2], sw_host[r % 2], stream=s_dn)
            srv_host[r % 2].copy_(srv_dev[r % 2], non_blocking=True)
    torch.cuda.synchronize()
    link_sw_ms = (time.perf_counter() - t_l) * 1e3 / 20
    S.sanns_set_response_primes(ctx, L)
    S.sanns_set_mac_sms(ctx, 0)
    # the host link alone: the same uploads and downloads, both directions at
    # once on their own streams, no compute
    link_reps = 20
    torch.cuda.synchronize()
    t_l = time.perf_counter()
    for r in range(link_reps):
        with torch.cuda.stream(s_up):
            ct_dev[r % 2].copy_(ct_host[r % nh:r % nh + 1], non_blocking=True)
        with torch.cuda.stream(s_dn):
            out_host[r % 2].copy_(out_dev[r % 2], non_blocking=True)
            srv_host[r % 2].copy_(srv_dev[r % 2], non_blocking=True)
    torch.cuda.synchronize()
    link_ms = (time.perf_counter() - t_l) * 1e3 / link_reps
    if dist:
        tt = torch.tensor([e2e_ms, e2e_seeded_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms, e2e_seeded_ms = float(tt[0].item()), float(tt[1].item())

    rb = _roofline_bytes(W)
    peak, peak_kind = _peaks()
    achieved = rb["total"] / (mac_avg * 1e-3) / 1e9
    ms_step = ms / args.steps
    value = world * n * args.steps / (ms * 1e-3)
    cpu = None
    if rank == 0:
        cpu = cpu_baseline_all_cores(quick=args.quick_cpu)
        cpu["single_core"] = cpu_baseline(quick=args.quick_cpu)
    batched = cluster = serving = alg4 = small = None
    if rank == 0 and not args.no_batched:
        del ct_all
        torch.cuda.empty_cache()
        batched = run_batched_section(quick=args.quick_batched)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_extra:
        small = run_small_section()
        cluster = run_cluster_section()
        torch.cuda.empty_cache()
        alg4 = run_alg4_section()
        torch.cuda.empty_cache()
        serving = run_serving_section()
        torch.cuda.empty_cache()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"linear scan, 1 query per step: n={n:,} d=128 uint8 "
                                   "64-component Gaussian mixture (sigma 20); BFV N=8192, three "
                                   "60-bit primes, t=16957441",
                       "n": n, "d": d, "N": N, "L": L, "K": K, "queries_cycled": W["n_queries"],
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "mac_variant": variant_names[variant],
                       "mac_variant_ms": dict(zip(variant_names, [round(x, 4) for x in variant_ms])),
                       "pipelining": "query s's MAC on stream A overlaps query s-1's INTT + mask "
                                     "on stream B (responses double-buffered); the MAC's grid "
                                     f"capped at {mac_sms or 'all'} SMs (tuned)",
                       "mac_sms_ms_per_step": {str(k): round(v, 4) for k, v in sms_ms.items()},
                       "pipelined_steps_bit_identical": pipe_exact,
                       "timed_steps": ("the K pipelined steps replayed from one captured CUDA graph" if use_graph
                                       else "the K pipelined steps issued from the host"),
                       "eager_ms_per_step": eager_ms / args.steps,
                       "eager_value": world * n / (eager_ms / args.steps * 1e-3),
                       "serial_ms_per_step": serial_ms,
                       "serial_mac_ms": serial_mac_ms,
                       "serial_mac_hbm_frac": rb["total"] / (serial_mac_ms * 1e-3) / 1e9 / peak,
                       "l2": "inputs larger than L2: the 3.1 GB encoded database is streamed "
                             "from HBM every step"},
            "latency_ms": {"p50": lat[len(lat) // 2],
                           "p99": lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]},
            "roofline": {"kernel": "mac_kernel (K2 ct x pt MAC)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": _mac_traffic(rb, W),
                         "traffic_source": "ncu capture at n = 200,000 scaled by blocks",
                         "algorithmic_bytes": rb["total"],
                         "launch_ms": mac_avg,
                         # in the timed loop the MAC's grid leaves SMs to the
                         # previous query's INTT + mask; alone on every SM:
                         "launch_sms": mac_sms or None,
                         "frac_alone_all_sms": rb["total"] / (serial_mac_ms * 1e-3) / 1e9 / peak},
            "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": d * 2 * L * N * 8,
                    "d2h_bytes_per_step": K * 2 * L * N * 8 + n * 4, "ms_per_step": e2e_ms,
                    "link_only_ms_per_step": link_ms,
                    "link_bound_frac": link_ms / e2e_ms,
                    "timing": "host wall clock over pipelined steps (4 streams: upload, MAC, "
                              "finish, download)"},
            "e2e_seeded_queries": {
                "value": world * n / (e2e_seeded_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": d * L * N * 8,
                "d2h_bytes_per_step": K * 2 * L * N * 8 + n * 4, "ms_per_step": e2e_seeded_ms,
                "rebuilt_ciphertext_bit_identical": seeded_exact,
                "what": "as e2e, but the client uploads c0 alone and the server rebuilds c1 from "
                        "the encryption seed (sanns_expand_query): an option beyond the paper, "
                        "whose client sends both components"},
            "e2e_switched_responses": {
                "value": world * n / (e2e_sw[False] * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": d * 2 * L * N * 8,
                "d2h_bytes_per_step": K * 2 * N * 8 + n * 4, "ms_per_step": e2e_sw[False],
                "shares_equal_brute_force": switched_exact,
                "seeded_queries": {"value": world * n / (e2e_sw[True] * 1e-3), "unit": UNIT,
                                   "h2d_bytes_per_step": d * L * N * 8,
                                   "d2h_bytes_per_step": K * 2 * N * 8 + n * 4,
                                   "ms_per_step": e2e_sw[True],
                                   "link_only_ms_per_step": link_sw_ms,
                                   "host_issue_ms_per_step": issue_sw[True]},
                "what": "as e2e, but the server switches each response down to q_0 "
                        "(sanns_set_response_primes; the client decrypts modulo q_0) and "
                        "downloads a third of the bytes: an option beyond the paper, whose "
                        "server sends the responses at the full modulus"},
            "selection": selection,
            "ntt": dict(_ntt_report(K * 2 * L, N, serial_fin_ms,
                                    "INTT + mask of one query (mask draw, intt_mask_short_kernel), "
                                    "on its own in the serial reference loop"),
                        overlapped_ms=fin_avg),
            "small_config": small,
            "ntt_form_responses": {"ms_per_step": nf_ms, "steps": cp_steps,
                                   "value": world * n / (nf_ms * 1e-3), "unit": UNIT},
            "slot_encoding": {"ms_per_step": sl_ms, "steps": cp_steps,
                              "value": world * n / (sl_ms * 1e-3), "unit": UNIT,
                              "shares_equal_brute_force": slot_exact},
            "circuit_privacy": {"ms_per_step": cp_ms, "flood_bits": flood, "steps": cp_steps,
                                "value": world * n / (cp_ms * 1e-3), "unit": UNIT,
                                "what": "public-key re-randomisation (one NTT per block per "
                                        "prime) + flooding e1 in [-2^F, 2^F) on c0, e2 on c1"},
            "cuda_graph": {"ms_per_step": graph_ms, "steps_per_graph": G, "replays": g_reps,
                           "pipelined_ms_per_step": ms_step,
                           "pipelined": "the main metric's timed steps (one graph of all of them)",
                           "value": world * n / (graph_ms * 1e-3), "unit": UNIT},
            "gpu_launches": 3 * args.steps,
            "clocks": ck,
            "cpu_baseline": cpu,
            "batched": batched,
            "clustering": cluster,
            "clustering_knns": alg4,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_gpu_sharded(args) -> None:
    """The linear-scan workload split across the ranks by block ranges
    (strong scaling: the total work is fixed).  Each rank encodes only its
    shard of the permuted point list (position base k0 N); per step rank 0's
    query ciphertext is broadcast over NCCL, every rank runs the distance step
    on its shard, and the response blocks and server shares are gathered back
    to rank 0, where they equal the single-GPU result bit for bit (checked on
    one step).  `e2e` adds rank 0's upload of the query from pinned host
    memory and its download of the gathered result."""
    import socket

    import torch
    import torch.distributed as dist

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S
    from paper_1904_02033_b300.shard import ShardDatabase, distances_sharded, shard_blocks

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world == 1 and "MASTER_PORT" not in os.environ:
        sk_ = socket.socket()
        sk_.bind(("127.0.0.1", 0))
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ["MASTER_PORT"] = str(sk_.getsockname()[1])
        sk_.close()
        os.environ.setdefault("RANK", "0")
        os.environ.setdefault("WORLD_SIZE", "1")
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOAD
    n, d, N, L = W["n"], W["d"], W["N"], W["L"]
    ctx = S.sanns_ctx_create(N, L, W["prime_bits"], W["t_rule"], d)
    coords = torch.from_numpy(inputs.mixture_coords(n, d, W["n_comp"], W["sigma"], W["seed"] + 1,
                                                    means_seed=W["seed"])).cuda()
    perm = torch.from_numpy(inputs.permutation(n, W["seed"] + 2)).cuda()
    K = -(-n // N)
    k0, k1 = shard_blocks(K, world, rank)
    shard = ShardDatabase(ctx, coords, perm, n, k0, k1)
    nq = W["n_queries"]
    qids = torch.arange(nq, dtype=torch.int64).to(torch.uint64).cuda()
    sk = S.sanns_keygen(ctx, W["seed"] + 3)
    queries = torch.from_numpy(inputs.mixture_coords(nq, d, W["n_comp"], W["sigma"], W["seed"] + 1001,
                                                     means_seed=W["seed"])).cuda()
    ct_all = S.sanns_encrypt_query(ctx, sk, queries, W["seed"] + 4, qids)   # used on rank 0 only
    buf = torch.empty((1, d, 2, L, N), dtype=torch.uint64, device="cuda")
    mask_seed = W["seed"] + 5
    state = {"qi": 0}

    def compute(ct_in, a, b):
        qi = state["qi"]
        return shard.distances(ct_in, mask_seed, qids[qi:qi + 1])

    def step(s):
        state["qi"] = s % nq
        if rank == 0:
            buf.copy_(ct_all[s % nq:s % nq + 1])
        return distances_sharded(compute, buf, n, N, L)

    # one step checked against the single-GPU run on rank 0
    res = step(0)
    exact = None
    if rank == 0:
        full = S.sanns_encode_db(ctx, coords, perm)
        o, sv = S.sanns_distances(ctx, full, ct_all[0:1], mask_seed, qids[0:1])
        exact = bool(torch.equal(res[0], o) and torch.equal(res[1], sv))
        del full, o, sv
    del res
    torch.cuda.empty_cache()
    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for s in range(args.steps):
        step(args.warmup + s)
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    tt = torch.tensor([ms], device="cuda")
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ms = float(tt.item())
    # end to end: rank 0 uploads the query from pinned memory and downloads
    # the gathered result every step
    ct_host = ct_all[:4].cpu().pin_memory() if rank == 0 else None
    out_host = torch.empty((1, K, 2, L, N), dtype=torch.uint64).pin_memory() if rank == 0 else None
    srv_host = torch.empty((1, n), dtype=torch.uint32).pin_memory() if rank == 0 else None
    e2e_steps = max(10, min(args.steps, 100))
    dist.barrier()
    torch.cuda.synchronize()
    tw = time.perf_counter()
    for s in range(e2e_steps):
        state["qi"] = s % nq
        if rank == 0:
            buf.copy_(ct_host[s % 4:s % 4 + 1], non_blocking=True)
        r = distances_sharded(compute, buf, n, N, L)
        if rank == 0:
            out_host.copy_(r[0], non_blocking=True)
            srv_host.copy_(r[1], non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - tw) * 1e3 / e2e_steps
    tt = torch.tensor([e2e_ms], device="cuda")
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_ms = float(tt.item())
    if rank == 0:
        line = {
            "metric": METRIC, "value": n * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"linear scan, 1 query per step, split over {world} GPU(s) by "
                                   f"block ranges: n={n:,} d=128 uint8 64-component Gaussian "
                                   "mixture (sigma 20); BFV N=8192, three 60-bit primes",
                       "n": n, "d": d, "N": N, "L": L, "K": K, "parallelism": f"blocks{world}",
                       "collectives": "NCCL broadcast of the query ciphertext from rank 0, gather "
                                      "of response blocks and server shares to rank 0",
                       "l2": "inputs larger than L2: each shard's encoded database is streamed "
                             "from HBM every step"},
            "gathered_result_equals_single_gpu": exact,
            "e2e": {"value": n / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": d * 2 * L * N * 8,
                    "d2h_bytes_per_step": K * 2 * L * N * 8 + n * 4},
            "gpu_launches": 3 * args.steps,
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


BATCHED = dict(n=10_000_000, d=96, N=8192, L=3, prime_bits=60, t_rule=0, n_comp=256, sigma=12.0,
               B=64, seed=7)


def run_batched_section(quick: bool = False, n_override: int | None = None,
                        d_override: int | None = None, b_override: int | None = None,
                        scratch_mib: int | None = None, tile: int | None = None) -> dict:
    """The batched configuration: n = 10^7, d = 96 (Deep1B-10M-shaped), 64
    queries per launch on the tensor-core path, against the same queries run
    one at a time on the per-query path; outputs compared in full."""
    import torch

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S

    W = dict(BATCHED)
    if quick:
        W["n"] = 1_000_000
    if n_override:
        W["n"] = n_override
    if d_override:
        W["d"] = d_override
    if b_override:
        W["B"] = b_override
    n, d, N, L, B = W["n"], W["d"], W["N"], W["L"], W["B"]
    ctx = S.sanns_ctx_create(N, L, W["prime_bits"], W["t_rule"], d)
    coords = inputs.mixture_coords_device(n, d, W["n_comp"], W["sigma"], W["seed"])
    perm = inputs.permutation_device(n, W["seed"] + 1)
    db = S.sanns_encode_db(ctx, coords, perm)
    del coords
    S.sanns_db_prepare_batched(ctx, db)
    q = inputs.mixture_coords_device(B, d, W["n_comp"], W["sigma"], W["seed"] + 2,
                                     means_seed=W["seed"])
    qids = torch.arange(B, dtype=torch.int64).to(torch.uint64).cuda()
    sk = S.sanns_keygen(ctx, W["seed"] + 3)
    ct = S.sanns_encrypt_query(ctx, sk, q, W["seed"] + 4, qids)
    K = db.K
    st = torch.cuda.current_stream()
    out_b = torch.empty((B, K, 2, L, N), dtype=torch.uint64, device="cuda")
    srv_b = torch.empty((B, n), dtype=torch.uint32, device="cuda")
    out_p = torch.empty((1, K, 2, L, N), dtype=torch.uint64, device="cuda")
    srv_p = torch.empty((1, n), dtype=torch.uint32, device="cuda")
    S.sanns_autotune_mac(ctx, db, ct[0:1], out_p, reps=2)
    if tile is not None:
        # a fixed tile shape (profiling captures), no autotuning
        S.sanns_batched_tune(ctx, scratch_mib=scratch_mib or 4096, tile=tile, prefetch_units=0)
        prefetch, tune_ms = 0, []
    else:
        if scratch_mib:
            S.sanns_batched_tune(ctx, scratch_mib=scratch_mib)
        tuned, tune_ms = S.sanns_autotune_batched(ctx, db, ct, out_b, reps=1)
        tile, prefetch = S.BATCHED_CONFIGS[tuned]

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # per-query path, the B queries one at a time
    def plain():
        for b in range(B):
            S.sanns_distances(ctx, db, ct[b:b + 1], 9, qids[b:b + 1], out_p, srv_p)
    t_plain = timed(plain, 1)
    # batched path, MAC stage alone then the whole step
    t_bmac = timed(lambda: S.sanns_distances_batched_mac(ctx, db, ct, out_b), 2)
    t_batch = timed(lambda: S.sanns_distances_batched(ctx, db, ct, 9, qids, out_b, srv_b), 2)
    S.sanns_device_status(ctx)
    # parity of the whole batch against the per-query path
    same = True
    for b in range(B):
        S.sanns_distances(ctx, db, ct[b:b + 1], 9, qids[b:b + 1], out_p, srv_p)
        same &= bool(torch.equal(out_p[0], out_b[b])) and bool(torch.equal(srv_p[0], srv_b[b]))
    # the same step with NTT-form responses (after the parity check, which
    # compares coefficient-form outputs)
    S.sanns_set_response_form(ctx, True)
    t_batch_ntt = timed(lambda: S.sanns_distances_batched(ctx, db, ct, 9, qids, out_b, srv_b), 2)
    t_plain_ntt = timed(plain, 1)
    S.sanns_device_status(ctx)
    S.sanns_set_response_form(ctx, False)
    flops = _batched_flops(B, K, d, L, N)
    peak = _peaks_tensor()
    rates = S.sanns_measure_mma_rates(ctx)
    int_rates = S.sanns_measure_int_rates(ctx)
    return {
        "workload": f"batched: n={n:,} d={d} uint8 256-component Gaussian mixture (sigma 12); "
                    f"{B} queries per launch; BFV N=8192, three 60-bit primes",
        "qp_per_s_batched": B * n / (t_batch * 1e-3),
        "qp_per_s_plain_per_query": B * n / (t_plain * 1e-3),
        "speedup_vs_plain": t_plain / t_batch,
        "ms_per_batch": t_batch, "ms_batched_mac": t_bmac, "ms_plain_for_B_queries": t_plain,
        "ntt_epilogue": dict(_ntt_report(B * K * 2 * L, N, t_batch - t_bmac,
                                         "fused INTT + mask (intt_mask_kernel), the batch's step minus its MAC stage"),
                             roofline=_ntt_roofline(int_rates, B * K * 2 * L, N, t_batch - t_bmac)),
        "ntt_form_responses": {"ms_per_batch": t_batch_ntt, "ms_plain_for_B_queries": t_plain_ntt,
                               "speedup_vs_plain": t_plain_ntt / t_batch_ntt,
                               "qp_per_s_batched": B * n / (t_batch_ntt * 1e-3)},
        "bit_identical_to_per_query_path": same,
        "autotuned": {"tile": ["128 blocks x 256 query rows per SM, producer-fed digits",
                               "256 blocks x 256 query rows per SM pair, producer-fed digits",
                               "128 blocks x 256 query rows per SM, TMA-fed fp16 digits",
                               "256 blocks x 256 query rows per SM pair, TMA-fed fp16 digits",
                               "128 blocks x 256 query rows per SM, TMA-fed, clusters of 2 sharing the query tile",
                               "128 blocks x 256 query rows per SM, TMA-fed, clusters of 4 sharing the query tile",
                               "128 blocks x 256 query rows per SM, TMA-fed, four slots per CTA, 32-byte stores",
                               "128 blocks x 256 query rows per SM, TMA-fed, four slots per CTA, 32-byte stores, "
                               "clusters of 2 sharing the query tile",
                               "256 blocks x 256 query rows per SM pair, TMA-fed, four slots per CTA pair, "
                               "32-byte stores"][tile],
                      "l2_prefetch_units": prefetch,
                      "ms_per_config": {f"tile{t}_prefetch{p}": round(m, 3)
                                        for (t, p), m in zip(S.BATCHED_CONFIGS, tune_ms)}},
        "roofline": {"kernel": "batched_mac_kernel (tcgen05 kind::f16, fp16 digits)",
                     "bound": "tensor", "achieved": flops / (t_bmac * 1e-3) / 1e12,
                     "peak": peak[0], "unit": "TFLOP/s",
                     "frac": flops / (t_bmac * 1e-3) / 1e12 / peak[0], "peak_source": peak[1],
                     "algorithmic_flops": flops},
        # raw instruction rates measured on this GPU by the library's probe:
        # fp16 digits on tcgen05 against the INT8 alternative (tcgen05 kind::i8
        # does not exist on sm_103a; legacy mma.sync s8 is what is left)
        "mma_rates": rates,
    }


CLUSTER = dict(n=1_000_000, d=128, N=8192, L=3, prime_bits=60, t_rule=0, k=1024, zipf=1.1,
               sigma=20.0, B=256, P=32, iters=20, seed=11)


def run_cluster_section() -> dict:
    """Clustering protocol: 1024 Lloyd clusters over Zipf(1.1)-weighted mixture
    data (n = 10^6, d = 128); 256 queries each probe their 32 nearest centres;
    all (query, block) work items of the batch run in one persistent launch."""
    import numpy as np
    import torch

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S

    W = CLUSTER
    n, d, N, L, B, Pr = W["n"], W["d"], W["N"], W["L"], W["B"], W["P"]
    ctx = S.sanns_ctx_create(N, L, W["prime_bits"], W["t_rule"], d)
    wts = inputs.zipf_weights(W["k"], W["zipf"])
    coords = inputs.mixture_coords_device_weighted(n, d, W["k"], W["sigma"], W["seed"], wts)
    centres, assign = inputs.lloyd_kmeans_device(coords, W["k"], W["iters"], W["seed"] + 1)
    order = torch.argsort(assign, stable=True).to(torch.int32).view(torch.uint32)
    cnt = torch.bincount(assign, minlength=W["k"]).cpu().numpy()
    offsets = np.zeros(W["k"] + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(cnt)
    cl = S.sanns_clusters_create(ctx, coords, offsets, order.contiguous())
    q = inputs.mixture_coords_device_weighted(B, d, W["k"], W["sigma"], W["seed"] + 2, wts,
                                              means_seed=W["seed"])
    probes = inputs.probes_device(q, centres, Pr).cpu().numpy().astype(np.uint32)
    qids = torch.arange(B, dtype=torch.int64).to(torch.uint64).cuda()
    sk = S.sanns_keygen(ctx, W["seed"] + 3)
    ct = S.sanns_encrypt_query(ctx, sk, q, W["seed"] + 4, qids)
    st = torch.cuda.current_stream()
    # warm-up, then timed launches
    out = S.sanns_distances_gather(ctx, cl, ct, probes, 5, qids)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        out = S.sanns_distances_gather(ctx, cl, ct, probes, 5, qids)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ct_out, srv, ids, n_b, k_b = out
    total_pts, total_blocks = int(n_b.sum()), int(k_b.sum())
    # the same query through the linear-scan entry point on its gathered list
    b = 0
    g = ids[: int(n_b[0])]
    db_b = S.sanns_encode_db(ctx, coords, g.contiguous())
    ref_out, ref_srv = S.sanns_distances(ctx, db_b, ct[0:1], 5, qids[0:1])
    same = bool(torch.equal(ref_out[0], ct_out[: int(k_b[0])])) and bool(
        torch.equal(ref_srv[0], srv[: int(n_b[0])]))
    S.sanns_device_status(ctx)
    # integer-pipe roofline: per work item d L forward transforms of the
    # gathered coordinates, 2 d L N modular multiply-adds (c0 and c1) and 2 L
    # inverse transforms, each transform N/2 log2 N butterflies; the ideal
    # time charges the forward butterflies and the multiply-adds at the
    # measured forward-butterfly rate and the inverse ones at the inverse rate
    rates = S.sanns_measure_int_rates(ctx)
    bf = N // 2 * (N.bit_length() - 1)
    fwd = total_blocks * W["d"] * W["L"] * bf
    macs = total_blocks * 2 * W["d"] * W["L"] * N
    inv = total_blocks * 2 * W["L"] * bf
    ideal_ms = ((fwd + macs) / rates["fwd_butterflies_per_s"] + inv / rates["inv_butterflies_per_s"]) * 1e3
    return {
        "roofline": {"kernel": "gather_kernel (K4: forward NTTs + MAC + INTT per work item)",
                     "bound": "alu", "achieved": (fwd + macs + inv) / (ms * 1e-3),
                     "peak": rates["fwd_butterflies_per_s"], "unit": "butterflies/s",
                     "frac": ideal_ms / ms, "ideal_ms": ideal_ms,
                     "peak_source": "library probe: register-resident butterflies on this GPU "
                                    "(sanns_measure_int_rates)",
                     "work": {"fwd_butterflies": fwd, "mac": macs, "inv_butterflies": inv},
                     "probe": rates},
        "workload": "clustering: n=1,000,000 d=128 uint8 mixture of 1024 Zipf(1.1)-weighted "
                    f"components (sigma 20); seeded Lloyd k-means to 1024 clusters; {B} queries x "
                    "32 probes; one persistent launch per batch; BFV N=8192, three 60-bit primes",
        "qp_per_s": total_pts / (ms * 1e-3),
        "ms_per_batch": ms, "queries": B, "gathered_points": total_pts,
        "work_items": total_blocks, "block_fill": total_pts / (total_blocks * N),
        "cluster_size_max_mean": [int(cnt.max()), float(cnt.mean())],
        "query0_bit_identical_to_linear_scan_on_its_gathered_list": same,
    }


ALG4 = dict(n=1_000_000, d=128, N=8192, L=3, prime_bits=60, t_rule=0, n_comp=64, sigma=20.0,
            m=20, alpha=0.56, s_max=31412, k=10, u=(50, 31, 19, 13), l=(458, 270, 178, 84),
            l_s=262, r_c=5, r_p=8, iters=3, B_lat=16, B_batch=64, seed=31)


def run_alg4_section() -> dict:
    """Algorithm 4 (clustering-based k-NNS) end to end through the library:
    balanced clustering (m = 20, alpha = 0.56) and a stash of at most 31,412
    points over n = 10^6, d = 128 mixture data, the SIFT row of the paper's
    hyperparameters (u^i, l^i, l_s, r_c, r_p); per-query latency, batched
    throughput and 10-NN accuracy against brute force."""
    import time

    import numpy as np
    import torch

    from paper_1904_02033_b300 import cluster, inputs
    from paper_1904_02033_b300 import sanns as S

    W = ALG4
    n, d = W["n"], W["d"]
    coords = inputs.mixture_coords_device(n, d, W["n_comp"], W["sigma"], W["seed"])
    t0 = time.perf_counter()
    groups = cluster.balanced_clustering(coords, W["m"], W["alpha"], iters=W["iters"], seed=W["seed"],
                                         max_search=3)
    kept, stash = cluster.split_stash(groups, W["s_max"])
    lay = cluster.make_layout(kept, stash, d, seed=W["seed"] + 1)
    t_cluster = time.perf_counter() - t0
    T = len(kept)
    u = tuple((list(W["u"]) + [W["u"][-1]] * T)[:T])
    l = tuple((list(W["l"]) + [W["l"][-1]] * T)[:T])
    ctx = S.sanns_ctx_create(W["N"], W["L"], W["prime_bits"], W["t_rule"], d)
    srv = cluster.ClusteringServer(ctx, coords, lay)
    sk = S.sanns_keygen(ctx, W["seed"] + 2)
    prm = cluster.Params(W["k"], u, l, W["l_s"], W["r_c"], W["r_p"])
    Bb = W["B_batch"]
    q_all = inputs.mixture_coords_device(Bb, d, W["n_comp"], W["sigma"], W["seed"] + 3,
                                         means_seed=W["seed"])
    qids = torch.arange(Bb, dtype=torch.int64).to(torch.uint64).cuda()
    cluster.query(srv, sk, q_all[:2], qids[:2], prm)       # warm-up
    torch.cuda.synchronize()
    lat = []
    for b in range(W["B_lat"]):
        t1 = time.perf_counter()
        cluster.query(srv, sk, q_all[b:b + 1], qids[b:b + 1], prm)
        lat.append((time.perf_counter() - t1) * 1e3)
    ids = cluster.query(srv, sk, q_all, qids, prm)            # warm-up at the batch size
    torch.cuda.synchronize()
    reps = 3
    t1 = time.perf_counter()
    for _ in range(reps):
        ids = cluster.query(srv, sk, q_all, qids, prm)
    batch_ms = (time.perf_counter() - t1) * 1e3 / reps
    # stage split (separate runs: each stage ends in a device synchronisation)
    st1, st64 = {}, {}
    for b in range(4):
        cluster.query(srv, sk, q_all[b:b + 1], qids[b:b + 1], prm, timings=st1)
    cluster.query(srv, sk, q_all, qids, prm, timings=st64)
    st1 = {key: round(v / 4, 3) for key, v in st1.items()}
    st64 = {key: round(v, 3) for key, v in st64.items()}
    # 10-NN accuracy against brute force (exact integer distances)
    xf = coords.to(torch.int64)
    kths = []
    for b in range(Bb):
        dq = ((xf - q_all[b].to(torch.int64)[None, :]) ** 2).sum(1)
        kths.append((dq, torch.kthvalue(dq, W["k"]).values))

    def accuracy(ids):
        a = 0.0
        for b in range(Bb):
            dq, kth = kths[b]
            got = torch.from_numpy(ids[b]).cuda()
            a += float(((dq[got.clamp(min=0)] <= kth) & (got >= 0)).sum()) / W["k"]
        return a / Bb

    acc = accuracy(ids)
    # the cost / accuracy trade-off: more clusters and bins per group
    sizes_g = np.diff(lay.group_offsets)
    tradeoff = []
    for scale in (2, 4, 8):
        us = tuple(int(min(x * scale, sizes_g[i])) for i, x in enumerate(u))
        ls = tuple(int(max(min(x * scale, sizes_g[i]), us[i])) for i, x in enumerate(l))
        p2 = cluster.Params(W["k"], us, ls, W["l_s"] * scale, W["r_c"], W["r_p"])
        cluster.query(srv, sk, q_all, qids, p2)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ids2 = cluster.query(srv, sk, q_all, qids, p2)
        ms2 = (time.perf_counter() - t2) * 1e3
        tradeoff.append({"u_l_scale": scale, "u": list(us), "ms_B64": ms2,
                         "queries_per_s": Bb / (ms2 * 1e-3), "accuracy_10nn": accuracy(ids2)})
    S.sanns_device_status(ctx)
    N = W["N"]
    sizes = np.diff(lay.cl_offsets.astype(np.int64))
    blocks = (-(-int(lay.group_offsets[-1]) // N) + -(-len(lay.stash_perm) // N)
              + -(-int(sum(u) * sizes.max()) // N))
    lat.sort()
    return {
        "workload": "Algorithm 4 (clustering-based k-NNS): n=1,000,000 d=128 uint8 64-component "
                    "Gaussian mixture (sigma 20); balanced clustering m=20 alpha=0.56 with stash; "
                    "u, l, l_s, r_c, r_p of the paper's SIFT row; BFV N=8192, three 60-bit primes",
        "groups": T, "centres_per_group": np.diff(lay.group_offsets).tolist(),
        "stash": len(lay.stash_perm), "cluster_size_max": int(sizes.max()),
        "u": list(u), "l": list(l), "clustering_s": t_cluster,
        "latency_ms_B1": {"p50": lat[len(lat) // 2], "max": lat[-1], "queries": len(lat)},
        "batch": {"queries": Bb, "ms": batch_ms, "queries_per_s": Bb / (batch_ms * 1e-3)},
        "stages_ms_B1": st1, "stages_ms_B64": st64,
        "response_blocks_per_query_at_most": blocks,
        "linear_scan_blocks_per_query": -(-n // N),
        "accuracy_10nn": acc,
        "tradeoff": tradeoff,
        "timing": "host wall clock per call (the pipeline reads selections back to plan the gather)",
    }


SERVE = dict(rate=2000.0, duration=10.0, max_batch=128, slots=2, mac_sms=128, seed=21, sample_frac=0.02)


def run_serving_section() -> dict:
    """Serving: Poisson arrivals at 2000 queries/s over two resident databases
    (n = 220,000, d = 50 and n = 10^6, d = 128, uint8 mixtures), continuous
    batching up to 128 queries, memory admission, p50/p99 latency."""
    import numpy as np
    import torch

    from paper_1904_02033_b300 import inputs
    from paper_1904_02033_b300 import sanns as S
    from paper_1904_02033_b300.serve import GpuExecutor, Request, Scheduler, run_open_loop

    W = SERVE
    specs = {"A": (220_000, 50, 64), "B": (1_000_000, 128, 64)}
    dbs, pools = {}, {}
    for i, (name, (n, d, ncomp)) in enumerate(specs.items()):
        ctx = S.sanns_ctx_create(8192, 3, 60, 0, d)
        coords = inputs.mixture_coords_device(n, d, ncomp, 20.0, 100 + i)
        db = S.sanns_encode_db(ctx, coords, inputs.permutation_device(n, 200 + i))
        S.sanns_db_prepare_batched(ctx, db)
        db.batched = True
        dbs[name] = (ctx, db)
        # a pool of client-encrypted queries, reused cyclically
        npool = 64
        q = inputs.mixture_coords_device(npool, d, ncomp, 20.0, 300 + i, means_seed=100 + i)
        qids = torch.arange(npool, dtype=torch.int64).to(torch.uint64).cuda()
        sk = S.sanns_keygen(ctx, 400 + i)
        pools[name] = (S.sanns_encrypt_query(ctx, sk, q, 500 + i, qids), qids)
    times = inputs.poisson_arrivals(W["rate"], W["duration"], W["seed"])
    # warm-up: one call per database on each path at the largest batch, so
    # the stream-ordered memory pool has grown before the timed runs
    for name, (ctx, db) in dbs.items():
        ct, qids = pools[name]
        reps = -(-W["max_batch"] // ct.shape[0])
        big = ct.repeat(reps, 1, 1, 1, 1)[:W["max_batch"]].contiguous()
        bq = torch.arange(W["max_batch"], dtype=torch.int64).to(torch.uint64).cuda()
        o, sv = S.sanns_distances_batched(ctx, db, big, 5, bq)
        del o, sv, big
        o, sv = S.sanns_distances(ctx, db, ct[0:1], 5, qids[0:1])
        del o, sv
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the per-query MAC leaves SMs free for another batch's INTT + mask on the
    # other slot's stream
    for ctx, _ in dbs.values():
        S.sanns_set_mac_sms(ctx, W["mac_sms"])
    # service times of both paths per database and batch size: each batch
    # then takes the faster path
    costs = GpuExecutor(dbs, slots=W["slots"], max_batch=W["max_batch"], batched_min=8).calibrate(pools)
    torch.cuda.empty_cache()

    def serve_once(window: float) -> dict:
        rnd = np.random.default_rng(W["seed"])
        reqs = []
        for rid, t in enumerate(times):
            name = "A" if rnd.random() < 0.5 else "B"
            ct, qids = pools[name]
            k = rid % ct.shape[0]
            reqs.append(Request(rid=rid, db=name, arrival=float(t),
                                payload=(ct[k:k + 1], qids[k:k + 1])))
        # the bit-exactness sample is drawn up front; only its requests keep
        # their responses on the device (a server hands each one off)
        sample = rnd.choice(len(reqs), size=max(1, int(W["sample_frac"] * len(reqs))), replace=False)
        sampled = {int(i) for i in sample}
        ex = GpuExecutor(dbs, slots=W["slots"], max_batch=W["max_batch"], batched_min=8,
                         keep=lambda r: r.rid in sampled)
        ex.costs = costs
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        sched = Scheduler(ex, max_batch=W["max_batch"], slots=W["slots"], mem_budget=int(free * 0.5),
                          batch_window=window)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = run_open_loop(sched, reqs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        # bit-exactness of the seeded sample: each result equals the query run alone
        exact = 0
        skipped = 0
        for i in sample:
            r = reqs[int(i)]
            if r.error is not None or r.result is None:   # rejected: nothing to compare
                skipped += 1
                continue
            ctx, db = dbs[r.db]
            o, sv = S.sanns_distances(ctx, db, r.payload[0], 5, r.payload[1])
            exact += int(torch.equal(o, r.result[0]) and torch.equal(sv, r.result[1]))
        pts = sum(specs[r.db][0] for r in reqs)
        sizes = [n for _, n, _ in stats.batches]
        return {
            "batch_window_ms": window * 1e3,
            "queries": len(reqs), "wall_s": wall, "qps": len(reqs) / wall,
            "qp_per_s": pts / wall,
            "latency_ms": {"p50": stats.percentile(50) * 1e3, "p99": stats.percentile(99) * 1e3},
            "batches": len(sizes), "mean_batch": float(np.mean(sizes)), "max_batch": int(max(sizes)),
            "tensor_path_batches": ex.tensor_batches,
            "tensor_path_queries": int(sum(n for (db, n, _) in stats.batches if ex.uses_tensor_path(db, n))),
            "deferred_for_memory": stats.deferred,
            "rejected_for_memory": stats.rejected,
            "mem_budget_bytes": sched.mem_budget,
            "sample_bit_exact": f"{exact}/{len(sample) - skipped}",
            "sample_skipped_rejected": skipped,
        }

    out = {"workload": "serving: Poisson 2000 q/s for 10 s over two resident databases "
                       "(n=220,000 d=50 and n=1,000,000 d=128), batches up to 128, 2 slots, "
                       "per-query MAC on 128 SMs, memory admission (library scratch included), "
                       "each batch on the path its calibrated service times favour"}
    out["service_ms"] = {db: {path: {str(b): round(ms, 3) for b, ms in tab} for path, tab in t.items()}
                         for db, t in costs.items()}
    out.update(serve_once(0.0))
    # the same arrivals with an 8 ms batching window: larger batches, which
    # take the tensor-core path (8 queries or more)
    out["batch_window_8ms"] = serve_once(0.008)
    return out


def _batched_flops(B: int, K: int, d: int, L: int, N: int) -> float:
    """Algorithmic FLOPs of one batched MAC: per (prime, slot) a GEMM with
    rows (query, component, query digit) = 2 B 8, columns the K blocks and a
    contraction over (dimension padded to a multiple of 8, database digit) =
    8 ceil(d / 8) 8, at 2 FLOPs per multiply-add."""
    dpad = (d + 7) // 8 * 8
    return 2.0 * (2 * B * 8) * K * (8 * dpad) * L * N


def _peaks_tensor():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), "measured bf16 dense (burst)"
    except Exception:
        return 1800.0, "fallback"


def _oracle_sample(n_blocks: int, n_queries: int):
    """Oracle setup for a bounded sample of the workload: the first n_blocks
    blocks of the database and n_queries encrypted queries."""
    from oracle.bfv import Oracle
    from paper_1904_02033_b300 import inputs

    W = WORKLOAD
    O = Oracle(W["N"], W["L"], W["prime_bits"], W["t_rule"], W["d"])
    npts = n_blocks * W["N"]
    coords = inputs.mixture_coords(npts, W["d"], W["n_comp"], W["sigma"], W["seed"] + 1,
                                   means_seed=W["seed"])
    queries = inputs.mixture_coords(n_queries, W["d"], W["n_comp"], W["sigma"], W["seed"] + 1,
                                    means_seed=W["seed"])
    _, s_hat = O.keygen(W["seed"] + 3)
    cts = [O.encrypt(s_hat, queries[i], W["seed"] + 4, i) for i in range(n_queries)]
    pt, norms = O.encode_db(coords, None)
    return O, pt, norms, cts, npts


def cpu_baseline(quick: bool = False) -> dict:
    """Time the oracle (single thread, as it stands) on a bounded sample: the
    MAC + INTT + mask of `blocks` database blocks for `queries` queries, with
    the sample's plaintexts encoded beforehand (untimed, like the resident
    database on the GPU)."""
    blocks, queries = (2, 1) if quick else (40, 2)
    O, pt, norms, cts, npts = _oracle_sample(blocks, queries)
    t0 = time.perf_counter()
    for ct in cts:
        acc = O.mac(ct, pt)
        O.intt_mask(acc, norms, npts, 0, blocks, WORKLOAD["seed"] + 5, 0)
    dt = time.perf_counter() - t0
    qp = npts * queries
    return {"value": qp / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{queries} queries x {blocks} blocks of 8192 points (d=128, N=8192, L=3): "
                      f"MAC + INTT + mask, {dt:.1f} s"}


def _cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo), for the baseline's record."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_all_cores(quick: bool = False) -> dict:
    """Time the oracle, as it stands, on every host core (at most 64): one
    thread per core, each running the single-threaded C loops (ctypes releases
    the GIL) on its own database blocks for the same encrypted queries.  The
    threads start together; the time is from the first start to the last end."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle.bfv import Oracle
    from paper_1904_02033_b300 import inputs

    W = WORKLOAD
    T = max(1, min(len(os.sched_getaffinity(0)), 64))
    bpt, nq = (1, 1) if quick else (2, 8)
    O = Oracle(W["N"], W["L"], W["prime_bits"], W["t_rule"], W["d"])
    npts = T * bpt * W["N"]
    coords = inputs.mixture_coords(npts, W["d"], W["n_comp"], W["sigma"], W["seed"] + 1,
                                   means_seed=W["seed"])
    queries = inputs.mixture_coords(nq, W["d"], W["n_comp"], W["sigma"], W["seed"] + 1,
                                    means_seed=W["seed"])
    _, s_hat = O.keygen(W["seed"] + 3)
    start = threading.Barrier(T, timeout=600)
    with ThreadPoolExecutor(T) as ex:
        cts = list(ex.map(lambda i: O.encrypt(s_hat, queries[i], W["seed"] + 4, i), range(nq)))
        enc = list(ex.map(lambda r: O.encode_db(coords, None, r * bpt, (r + 1) * bpt), range(T)))

        def work(r):
            pt, norms = enc[r]
            start.wait()
            t0 = time.perf_counter()
            for i, ct in enumerate(cts):
                acc = O.mac(ct, pt)
                O.intt_mask(acc, norms, npts, r * bpt, (r + 1) * bpt, W["seed"] + 5, i)
            return t0, time.perf_counter()

        spans = list(ex.map(work, range(T)))
    dt = max(e for _, e in spans) - min(b for b, _ in spans)
    return {"value": npts * nq / dt, "unit": UNIT, "cores": T, "kind": "oracle",
            "cpu": _cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{T} threads x {bpt} blocks of 8192 points each, {nq} queries "
                      f"(d=128, N=8192, L=3): MAC + INTT + mask, {dt:.1f} s"}


def run_reference(args) -> None:
    """The oracle as it stands on every host core (at most 64 threads, the C
    loops run without the GIL): each step, every thread takes one query's MAC
    + INTT + mask over its own database block."""
    from concurrent.futures import ThreadPoolExecutor

    rank, world, _ = _env_rank()
    if rank != 0:
        return
    T = max(1, min(len(os.sched_getaffinity(0)), 64))
    O, pt, norms, cts, npts = _oracle_sample(T, 1)
    ct = cts[0]
    N = WORKLOAD["N"]

    def block(r):
        acc = O.mac(ct, pt[r:r + 1])
        O.intt_mask(acc, norms[r * N:(r + 1) * N], npts, r, r + 1, WORKLOAD["seed"] + 5, 0)

    with ThreadPoolExecutor(T) as ex:
        def step():
            list(ex.map(block, range(T)))

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t0
    value = npts * args.steps / dt
    sample = (f"per step 1 query x {T} blocks of 8192 points (d=128, N=8192, L=3), one block per "
              f"thread: MAC + INTT + mask")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "linear scan, 1 query per step: n=1,000,000 d=128 uint8 "
                               "64-component Gaussian mixture (sigma 20); BFV N=8192, three "
                               "60-bit primes, t=16957441 (CPU oracle on a bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": T, "kind": "oracle",
                         "cpu": _cpu_model(), "nproc": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="sanns", choices=["sanns", "reference"])
    ap.add_argument("--quick-cpu", action="store_true", help="smaller CPU baseline sample")
    ap.add_argument("--mac-variant", default=None, help="fixed MAC launch variant instead of the autotuner's")
    ap.add_argument("--mac-sms", type=int, default=None, help="fixed MAC SM cap instead of the tuned one")
    ap.add_argument("--shard", action="store_true",
                    help="split the linear-scan database across the ranks by block ranges "
                         "(broadcast + gather) instead of running replicas")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched section")
    ap.add_argument("--no-extra", action="store_true", help="skip the clustering and serving sections")
    ap.add_argument("--only", choices=["cluster", "serving", "alg4"], default=None,
                    help="run only one of the extra sections")
    ap.add_argument("--quick-batched", action="store_true", help="batched section at n = 10^6")
    ap.add_argument("--only-batched", type=int, default=None, metavar="N_POINTS",
                    help="run only the batched section on N_POINTS points (profiling)")
    ap.add_argument("--batched-d", type=int, default=None, help="dimension for --only-batched")
    ap.add_argument("--batched-B", type=int, default=None, help="queries per launch for --only-batched")
    ap.add_argument("--batched-tile", type=int, default=None, choices=list(range(9)),
                    help="fixed tile shape of the batched MAC for --only-batched (no autotuning)")
    ap.add_argument("--batched-scratch-mib", type=int, default=None,
                    help="cap on the batched path's query-multiple scratch (smaller launches)")
    ap.add_argument("--n", type=int, default=None,
                    help="smaller database (profiling captures); the line then names it")
    ap.add_argument("--queries", type=int, default=None, help="number of distinct queries")
    ap.add_argument("--cluster-B", type=int, default=None,
                    help="queries per batch in the clustering section (profiling captures)")
    args = ap.parse_args()
    if args.n is not None:
        WORKLOAD["n"] = args.n
    if args.queries is not None:
        WORKLOAD["n_queries"] = args.queries
    if args.cluster_B is not None:
        CLUSTER["B"] = args.cluster_B
    if args.warmup < 3:
        args.warmup = 3
    if args.only:
        import torch
        torch.cuda.set_device(0)
        fn = {"cluster": run_cluster_section, "serving": run_serving_section,
              "alg4": run_alg4_section}[args.only]
        print(json.dumps({args.only: fn()}), flush=True)
    elif args.only_batched:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"batched": run_batched_section(n_override=args.only_batched,
                                                         d_override=args.batched_d,
                                                         b_override=args.batched_B,
                                                         scratch_mib=args.batched_scratch_mib,
                                                         tile=args.batched_tile)}),
              flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_gpu_sharded(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

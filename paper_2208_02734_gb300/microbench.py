"""Run one MASK step on seeded synthetic data and time it (CUDA events).

Used to look at a single kernel in isolation (e.g. under a profiler):

  python -m paper_2208_02734_gb300.microbench assign --n 1000000 --d 64 --k 4096
  python -m paper_2208_02734_gb300.microbench update --n 1000000 --d 64 --k 4096
  python -m paper_2208_02734_gb300.microbench kmeanspp --n 262144 --d 64 --k 2048
  python -m paper_2208_02734_gb300.microbench query --n 1000000 --d 64 --k 4096 \
      --levels 4096,128 --probes 64,16 --nq 10000
  python -m paper_2208_02734_gb300.microbench csr_assign --n 200000 --d 20000 --k 4096
  python -m paper_2208_02734_gb300.microbench csr_kmeanspp --n 200000 --d 20000 --k 512
  python -m paper_2208_02734_gb300.microbench csr_query --n 200000 --d 20000 --k 4096 \
      --levels 1024,64 --probes 64,16 --nq 2000

The csr_* steps use CSR rows from synth.sparse_tfidf_like (log-normal lengths
of mean 60, Zipf column ids, unit rows).

Dense points come from an anisotropic Gaussian mixture
(synth.AnisotropicMixture, 100 blobs); prints one JSON line with the mean time
per call.
"""

from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("step", choices=["assign", "update", "kmeanspp", "query", "build",
                                     "csr_assign", "csr_kmeanspp", "csr_query", "csr_build",
                                     "mma_probe"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=64)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--levels", type=str, default="")
    ap.add_argument("--probes", type=str, default="")
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--topk", type=int, default=10)
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="fp32",
                    help="query step: the leaf scan's precision")
    ap.add_argument("--profile", action="store_true",
                    help="also report the library's per-kernel device times")
    a = ap.parse_args(argv)

    import torch

    from . import mask as M
    from . import synth

    dev = torch.device("cuda:0")
    if a.step == "mma_probe":
        # cycles per tcgen05 kind::f16 MMA (M = 128, K = 16) by N, operand A's
        # memory and the number of accumulators used round-robin
        torch.cuda.init()
        rounds = 256
        for n in (64, 128, 192, 256):
            for a_tmem in (False, True):
                for n_acc in (1, 2):
                    if n_acc * n > (448 if a_tmem else 512):
                        continue
                    issue, done = M.mask_test_tc_mma_cycles(n, a_tmem, n_acc, rounds)
                    mmas = 12 * rounds
                    print(json.dumps({"step": "mma_probe", "n": n, "a": "tmem" if a_tmem else "smem",
                                      "n_acc": n_acc, "cycles_per_mma": round(done / mmas, 1),
                                      "issue_cycles_per_mma": round(issue / mmas, 1),
                                      "f16_mac_per_cycle": round(128 * n * 16 * mmas / done)}),
                          flush=True)
        return
    levels = [int(v) for v in a.levels.split(",")] if a.levels else [a.k]
    probes = [int(v) for v in a.probes.split(",")] if a.probes else [8] * len(levels)
    rng = np.random.default_rng(1)
    state = {}
    if a.step.startswith("csr_"):
        A = synth.sparse_tfidf_like(a.n, a.d, seed=0)
        csr = tuple(torch.from_numpy(x).to(dev) for x in (A.row_ptr, A.col, A.val))
        rows = rng.choice(a.n, a.k, replace=False)
        C = torch.from_numpy(A.rows(rows).to_dense(np.float32)).to(dev)
        if a.step == "csr_query":
            Qa = synth.sparse_tfidf_like(a.nq, a.d, seed=1)
            state["Q"] = tuple(torch.from_numpy(x).to(dev) for x in (Qa.row_ptr, Qa.col, Qa.val))
            state["index"] = M.mask_build_csr(*csr, a.d, levels, a.iters, seed=0)
    else:
        mix = synth.AnisotropicMixture(d=a.d, n_blobs=100, seed=0)
        X = torch.from_numpy(mix.sample(a.n, seed=0)).to(dev)
        C = X[torch.from_numpy(rng.choice(a.n, a.k, replace=False)).to(dev)].contiguous()

    if a.step == "update":
        state["labels"], _ = M.mask_kmeans_assign(X, C, with_dist=False)
    if a.step == "query":
        state["index"] = M.mask_build(X, levels, a.iters, seed=0)
        state["Q"] = torch.from_numpy(mix.sample(a.nq, seed=1)).to(dev)

    def run():
        if a.step == "assign":
            M.mask_kmeans_assign(X, C, with_dist=False)
        elif a.step == "update":
            M.mask_kmeans_update(X, state["labels"], C)
        elif a.step == "kmeanspp":
            M.mask_kmeanspp(X, a.k, seed=0)
        elif a.step == "query":
            prec = {"fp32": M.MASK_FP32, "bf16": M.MASK_BF16, "fp8": M.MASK_FP8E4M3}[a.precision]
            M.mask_query(state["index"], state["Q"], a.topk, probes, precision=prec)
        elif a.step == "csr_assign":
            M.mask_kmeans_assign_csr(*csr, a.d, C, with_dist=False)
        elif a.step == "csr_kmeanspp":
            M.mask_kmeanspp_csr(*csr, a.d, a.k, seed=0)
        elif a.step == "csr_query":
            M.mask_query_csr(state["index"], *state["Q"], a.topk, probes)
        elif a.step == "csr_build":
            M.mask_build_csr(*csr, a.d, levels, a.iters, seed=0).free()
        else:
            M.mask_build(X, levels, a.iters, seed=0).free()

    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    if a.profile:
        M.mask_profile_reset()
        M.mask_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    out = {"step": a.step, "n": a.n, "d": a.d, "k": a.k, "ms": ms}
    if a.profile:
        M.mask_profile_enable(False)
        for name in ("assign_tc", "assign_gemm", "assign_recheck", "kmeanspp", "label_sort",
                     "centroid_update", "scan_topk_level", "scan_topk_leaf", "scan_leaf_cm",
                     "leaf_group", "leaf_merge", "scan_leaf_bf16", "scan_leaf_fp8", "leaf_rerank",
                     "csr_scan_leaf_cm", "csr_assign",
                     "csr_spmm_assign", "csr_centroid_update", "csr_scan_level", "csr_scan_leaf"):
            r = M.mask_profile_read(name)
            if r:
                out[name + "_ms"] = r[1] / max(1, r[0])
    if a.step == "assign":
        out["tflops"] = 2.0 * a.n * a.k * a.d / (ms / 1e3) / 1e12
        kms = out.get("assign_tc_ms") or out.get("assign_gemm_ms")
        if kms:
            out["kernel_tflops"] = 2.0 * a.n * a.k * a.d / (kms / 1e3) / 1e12
    if a.profile and "assign_tc_ms" in out:
        r = M.mask_profile_read("assign_tc")
        out["assign_tc_useful_tflops"] = r[2] / max(1, r[0]) / (out["assign_tc_ms"] / 1e3) / 1e12
    if a.step == "csr_assign" and "csr_spmm_assign_ms" in out:
        r = M.mask_profile_read("csr_spmm_assign")
        out["spmm_tflops"] = r[2] / max(1, r[0]) / (out["csr_spmm_assign_ms"] / 1e3) / 1e12
    if a.step in ("csr_kmeanspp",) and "kmeanspp_ms" in out:
        r = M.mask_profile_read("kmeanspp")
        out["kpp_gbs"] = r[2] / max(1, r[0]) / (out["kmeanspp_ms"] / 1e3) / 1e9
    if a.step in ("kmeanspp", "csr_kmeanspp") and "kmeanspp_ms" in out:
        out["kpp_us_per_step"] = out["kmeanspp_ms"] * 1e3 / max(1, a.k - 1)
    print(json.dumps(out))
    if "index" in state:
        state["index"].free()


if __name__ == "__main__":
    main()

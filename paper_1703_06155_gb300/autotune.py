"""Autotuner of the run-time tunables of a context (h2_set_opts).

For one workload (a built context and its right-hand sides) it times the
step a user repeats -- factorization plus refined solve -- with CUDA events
for candidate settings of

  tile_policy   batched-GEMM tile shape rule (least padded work / 64-wide),
  split_target  CTAs a GEMM launch is split-K'ed up to,
  cluster_max   CTAs per Step-0 subspace / eigen problem,
  apply_path    Step-2 and panel applications (GEMM + copy / in place),
  tensor_cores  complex64 tiles on tcgen05 / warp-level tensor-core MMAs
                (3xTF32) or on FP32 FMAs,
  gram_emulation  FP64-accurate Step-0 Grams on the FP32 pipe / FP64 FMAs,
  eig_solver    Step-0 eigen-decomposition: cyclic Jacobi / tridiagonal + QL /
                one-sided Jacobi SVD of the Cholesky factor,
  stop_level    early stop of the factorization (Sec. III-C): l0 (0) or one
                to three levels below it, the rest as one dense final block,
  ldlt          block LDL^T in FP64 only / in both precisions (symmetric
                matrices; block LU otherwise),

one parameter at a time from the defaults (coordinate descent), keeps the
fastest setting of each and leaves it set on the context.  Every timing runs
in the library; this module only chooses among them.
"""
import torch

DEFAULT_SPACE = {
    "tensor_cores": [2, 1, 0],
    "gram_emulation": [1, 0],
    "tile_policy": [0, 1],
    "split_target": [0, 608, 2432],
    "cluster_max": [16, 8],
    "apply_path": [2, 1],
    "eig_solver": [2, 0, 1],
    "ldlt": [2, 1],
}


def stop_levels(ctx, extra=3):
    """Candidate stop levels of a context: 0 (= l0) and l0 + 1 .. l0 + extra (<= L)."""
    L, l0 = ctx._sizes()[1:3]
    return [0] + [s for s in range(l0 + 1, min(L, l0 + extra) + 1)]


def _time_step(ctx, b, eps, precision, tol, stream, repeats):
    ctx.factorize(eps, precision)  # warm-up (arenas sized)
    ctx.solve(b, refine=True, tol=tol, max_iter=30, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        ctx.factorize(eps, precision)
        ctx.solve(b, refine=True, tol=tol, max_iter=30, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats


def autotune(ctx, b, eps, precision="mixed", tol=1e-6, space=None, repeats=2, stream=None, profile=0):
    """Returns (best settings, list of (settings, ms per step)); the best
    settings are left applied to `ctx`."""
    if space is None:
        space = dict(DEFAULT_SPACE)
        space["stop_level"] = stop_levels(ctx)
        if not ctx.stats()["symmetric"]:
            space["ldlt"] = [2]  # block LU either way: the LDL^T form needs a symmetric matrix
    space = dict(space)
    stream = stream or torch.cuda.current_stream()
    best = {k: v[0] for k, v in space.items()}
    log = []

    def run(cfg):
        ctx.set_opts(profile=profile, **cfg)
        ms = _time_step(ctx, b, eps, precision, tol, stream, repeats)
        log.append((dict(cfg), ms))
        return ms

    best_ms = run(best)
    for key, values in space.items():
        for v in values:
            if v == best[key]:
                continue
            cfg = dict(best, **{key: v})
            ms = run(cfg)
            if ms < best_ms:
                best_ms, best = ms, cfg
    ctx.set_opts(profile=profile, **best)
    return best, log

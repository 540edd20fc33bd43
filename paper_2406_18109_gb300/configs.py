"""Workload configurations (sizes, seeds and launch settings) shared by the
benchmark, the smoke check and the full-size parity tests, so that the tests
check exactly the launch configuration the benchmark times.  Launch settings
(block, unroll, tile, rows) were chosen by sweeping them on a GB300."""

# Black-Scholes: 2^26 FP32 options (spot U[5,30], strike U[1,100], expiry
# U[0.25,10], r = 0.02, sigma = 0.3, seed 1)
BLACK_SCHOLES = dict(n=1 << 26, seed=1, r=0.02, sigma=0.3, tile=16384, block=1024, unroll=2,
                     # ncu counters of the fused kernel named `kernel` (generated
                     # kernels are named by a hash of their code, so a change to
                     # the generated code changes the name and retires them):
                     # thread instructions per option (smsp__inst_executed x 32
                     # / options; the kernel is bound by instruction issue) and
                     # DRAM bytes (read + write) of one launch at n = 2^26
                     counters=dict(kernel="dfs_k62b33cd1f6ebfe5d", inst_per_option=111.91,
                                   dram_bytes_per_launch=1301.96e6),
                     # end to end (host arrays): kernels on mapped host memory
                     # ("zero_copy") or copies pipelined in chunks over contexts
                     e2e_mode="zero_copy", e2e_chunk=1 << 23, e2e_contexts=2)

# CG: 2-D 5-point Poisson on a 256x256 grid, 50 iterations, FP64 values,
# int32 indices, x* ~ U[-1,1] (seed 0), b = A x*, x0 = 0; five iterations
# share one flush window (one persistent launch) in the captured solve
CG = dict(m=256, iters=50, seed=0, tile=512, block=256, unroll=1, iters_per_flush=5, window_size=1024,
          # ncu counters of the steady five-iteration window kernel named
          # `kernel` (this launch shape): DRAM bytes per iteration; the rest of
          # the traffic is served by L2 (profiles/)
          counters=dict(kernel="dfs_kd2a6167401cf8ba5", dram_bytes_per_iteration=5.851904e6 / 5))

# Batched CG: 256 independent solves of uneven size (half 2-D Poisson with m
# log-uniform in [32, 1024], half random diagonally dominant SPD with n
# log-uniform in [1024, 65536]), 100 iterations each, one batched launch per
# iteration, the whole solve replayed from a CUDA graph; FP64 (dtype "f32"
# for the FP32 variant).  Tiles follow the size-dependent policy (at least two
# points per problem, at most tile_max elements); the bench autotunes
# tile_max and the launch shape before capturing.
BATCHED_CG = dict(count=256, seed=4, iters=100, dtype="f64", tile_max=2048, min_points=2, block=256, unroll=2,
                  # ncu counters of the batched iteration kernel named `kernel`,
                  # FP64 and FP32, at this launch shape: DRAM bytes (read + write)
                  # per launch (profiles/)
                  counters=[dict(kernel="dfs_b0fc715b3e5f18a2c", dram_bytes_per_launch=3.019141e9 + 0.672542e9),
                            dict(kernel="dfs_b0a54bf6785d3c28c", dram_bytes_per_launch=1.865591e9 + 0.315713e9)])

# Jacobi: Fig. 1 stencil on an 8192x8192 FP32 grid (8190^2 interior),
# 200 sweeps, interior U[0,1] (seed 2), boundary 1.0
JACOBI = dict(N=8190, sweeps=200, seed=2, rows=16, block=512, unroll=4, sweeps_per_flush=1,
              # ncu counters (one-pass metrics, full size) of the sweep kernel
              # named `kernel`: DRAM bytes (read + write) of one launch (one sweep)
              counters=dict(kernel="dfs_ka23239f399de85c0", dram_bytes_per_launch=540.48e6 + 487.56e6))

# Serving: Poisson arrivals (exponential gaps, mean 2 ms, seed 3) of CG and
# BiCGSTAB solves on 3-D 7-point Poisson operators (m from a log-spaced
# ladder 64..256, FP64, tol 1e-8) and Black-Scholes batches of 2^16..2^24
# FP32 options, under a 120 GB device-memory budget; solves advance 8
# iterations per tick; at most 64 active solves per kind.  `count` requests
# per run (a bounded stand-in for an open-ended stream).
SERVING = dict(count=240, seed=3, mean_gap_ms=2.0, budget_gb=120, tol=1e-8, iters_per_tick=8, max_active=64,
               tile=4096, block=256, unroll=2, load_fraction=0.8)

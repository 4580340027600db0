/*
 * mppi_serve.h - batched serving of many independent MPPI problems (C ABI).
 *
 * The paper runs one controller per robot (Sec. IV-A).  This layer serves
 * many independent problems of uneven size (K samples, T steps) from one GPU:
 *   - problems are registered once; their nominal plans stay on the device
 *     and are warm-started by their own updates (Sec. II, last paragraph);
 *   - requests (one MPPI update of one problem from a given state) are
 *     queued; a scheduler batches every admissible request into a tick and
 *     runs the tick as ONE CUDA-graph launch of two persistent kernels
 *     (rollout tiles of all problems, then the Eq. 4 update entries of all
 *     problems), identical per sample to the single-problem path;
 *   - admission is by memory: a request needs 4 K (7 T + 1) bytes of scratch
 *     (costs and noise) from a fixed device pool and waits, in arrival order,
 *     until that much is free; scratch returns to the pool when its tick ends;
 *   - up to `lanes` ticks are in flight at once on separate streams, so work
 *     of requests that arrive while a tick runs overlaps with it on the GPU
 *     (continuous batching); requests of one problem run one after another;
 *   - an autotuner times the rollout kernel variants and tile sizes on the
 *     registered mix and keeps the fastest.
 * Status codes and error messages follow mppi.h.  All calls are thread-safe
 * except create/destroy.
 */
#ifndef MPPI_SERVE_H
#define MPPI_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "mppi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- device memory pool (host-side bookkeeping, no CUDA) ----------------
 * First-fit allocator over [0, bytes) with 256-byte granularity and
 * coalescing of free neighbours; the server uses it for request scratch. */
typedef struct mppi_pool_s* mppi_pool_t;
MPPI_API int mppi_pool_create(size_t bytes, mppi_pool_t* out);
MPPI_API int mppi_pool_destroy(mppi_pool_t pool);
/* MPPI_ERR_OOM when no free block fits; offsets are multiples of 256. */
MPPI_API int mppi_pool_alloc(mppi_pool_t pool, size_t bytes, size_t* offset);
/* MPPI_ERR_INVALID_ARG if offset is not the start of a live allocation. */
MPPI_API int mppi_pool_free(mppi_pool_t pool, size_t offset);
/* out: size, bytes in use, peak bytes in use, largest free block. */
MPPI_API int mppi_pool_stats(mppi_pool_t pool, size_t out[4]);

/* ---- server ---------------------------------------------------------- */
typedef struct mppi_server_s* mppi_server_t;

typedef struct mppi_server_config {
  size_t pool_bytes;  /* device bytes for request scratch                    */
  int max_problems;   /* registered problems, 1..4096                         */
  int max_batch;      /* requests per tick, 1..1024                           */
  int lanes;          /* ticks in flight at once, 1..4                        */
  int variant;        /* rollout kernel: 0 autotune (unrolled until tuned),
                         1 unrolled, 2 rolled, 3 warp-specialised (tiles of
                         32 samples on 96 threads)                            */
  int rollout_block;  /* samples per tile for variants 1, 2: 0 autotune, or
                         32, 64, 128                                          */
} mppi_server_config;

/* Creates the server on the current device: allocates the pool, the problem
 * table and per-lane streams and descriptors. */
MPPI_API int mppi_server_create(const mppi_server_config* cfg, mppi_server_t* out);
/* Stops the scheduler, waits for in-flight ticks, frees everything. */
MPPI_API int mppi_server_destroy(mppi_server_t srv);

/* Registers a problem (arm, cost, sizes and sampler as for mppi_create; the
 * reduction is FP32).  Its plan starts at zero and its iter at 0.  *id is
 * the problem's handle.  MPPI_ERR_OOM if the problem table is full or its
 * scratch could never fit in the pool. */
MPPI_API int mppi_server_add_problem(mppi_server_t srv, const mppi_robot* robot,
                                     const mppi_cost* cost, const mppi_config* cfg, int* id);
/* Plan of a problem ([T][7], host); set is refused while it has work queued
 * or in flight (MPPI_ERR_INVALID_ARG). */
MPPI_API int mppi_server_set_plan(mppi_server_t srv, int id, const float* u);
MPPI_API int mppi_server_get_plan(mppi_server_t srv, int id, float* u);
MPPI_API int mppi_server_get_iter(mppi_server_t srv, int id, uint64_t* iter);

/* Queues one update of problem id from the 25 input floats (q, qd, goal,
 * plane as in mppi_step_device, host memory, copied).  *ticket identifies it. */
MPPI_API int mppi_server_submit(mppi_server_t srv, int id, const float in[25], uint64_t* ticket);
/* *done = 1 and tau0 filled (if not NULL) when the request has finished;
 * returns the request's status (MPPI_OK or MPPI_ERR_NONFINITE) or, while it
 * is pending, MPPI_OK with *done = 0.  A finished ticket can be polled once. */
MPPI_API int mppi_server_poll(mppi_server_t srv, uint64_t ticket, float tau0[7], int* done);
/* Blocks until the request has finished; as poll otherwise. */
MPPI_API int mppi_server_wait(mppi_server_t srv, uint64_t ticket, float tau0[7]);

/* Background scheduler thread (continuous batching) on/off.  While ticks
 * are in flight, and for 2 ms after its last tick or request, the thread
 * polls (yielding its core) rather than sleeping, so that new requests are
 * admitted without a thread wake-up; after that it sleeps until a request
 * arrives. */
MPPI_API int mppi_server_start(mppi_server_t srv);
MPPI_API int mppi_server_stop(mppi_server_t srv);
/* One scheduling round from the calling thread, for use without the thread:
 * retires finished ticks, then launches at most one new tick.  *launched
 * receives the number of requests in the new tick (0 if none). */
MPPI_API int mppi_server_tick(mppi_server_t srv, int* launched);
/* Blocks until nothing is queued or in flight (runs rounds itself when the
 * scheduler thread is not running). */
MPPI_API int mppi_server_drain(mppi_server_t srv);

/* Times every (variant, tile size) on one tick holding one request of each
 * registered problem (up to max_batch; plans and iters are not changed) and
 * keeps the fastest; *best_ms receives its rollout time.  Needs an idle
 * server with the scheduler thread stopped. */
MPPI_API int mppi_server_autotune(mppi_server_t srv, float* best_ms);

/* out: requests completed, ticks launched, mean requests per tick, peak
 * pool bytes, pool bytes, chosen variant, chosen tile size, rollout-steps
 * completed. */
MPPI_API int mppi_server_stats(mppi_server_t srv, double out[8]);

/* Native open-loop load test: Poisson arrivals at rate_hz for `seconds`,
 * each an update of a uniformly chosen registered problem from the inputs
 * last given with mppi_server_set_input; needs the scheduler thread running.
 * out: completed, p50 latency [ms], p99 latency [ms], mean latency [ms],
 * throughput [updates/s], rollout-steps/s, mean requests per tick, max
 * queue length. Latency is completion minus arrival. */
MPPI_API int mppi_server_set_input(mppi_server_t srv, int id, const float in[25]);
MPPI_API int mppi_server_load_test(mppi_server_t srv, double rate_hz, double seconds,
                                   uint64_t seed, double out[8]);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_SERVE_H */

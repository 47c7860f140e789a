// Hooks of the grid object for the batch and serving runtime (rmt_batch.cu); not part of the
// C ABI.
#pragma once
#include <cuda_runtime.h>

#include "rmt.h"

struct MGSolver;

// Makes g a member of a batch launched on batch_stream: initialises it, checks that a step
// has no host synchronisation (fixed multigrid cycles, profiling off) and waits for its stream.
rmt_status grid_join_batch(rmt_grid* g, cudaStream_t batch_stream);
void grid_leave_batch(rmt_grid* g);
// Records one step of g on s (a stream in capture); g's host state is left unchanged.
rmt_status grid_capture_step(rmt_grid* g, cudaStream_t s);
// The host state after one step that ran from a captured graph (parity, time, step count).
void grid_advance_host(rmt_grid* g);
int grid_parity(const rmt_grid* g);
// Waits for g's stream and reads its device error words (degenerate fits, non-finite values).
rmt_status grid_check(rmt_grid* g);
// The same without waiting: the error words as of the last step whose copy has landed.
rmt_status grid_poll(rmt_grid* g);
// Host-side work before a batched step of g, enqueued on s (the fault injection of the
// inject_nan_step option).
rmt_status grid_pre_step(rmt_grid* g, cudaStream_t s);
// Records an error on g (sticky unless RMT_EINVAL).
rmt_status grid_fail(rmt_grid* g, rmt_status st, const char* msg);
// The grid's two multigrid solvers and stream, for the autotuner; RMT_ESTATE before the first
// step (the solvers' right-hand sides are those of the last step).
rmt_status grid_solvers(rmt_grid* g, MGSolver** mac, MGSolver** fe, cudaStream_t* s, double* rtol);

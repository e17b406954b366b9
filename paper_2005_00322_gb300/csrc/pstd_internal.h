// pstd_internal.h -- plan internals shared by the batch layer (not exported).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pstd.h"

// Launch `n` leapfrog steps of plan P on its own stream (no graph capture of
// its own, so the caller may be capturing); adds the kernel count.
int pstd_internal_launch_steps(pstd_plan_t* P, float* p, float* const* u, int64_t n, int64_t* launches);
// Convert the register-FFT axes' velocities of plan P in place to their
// spectrum form (to_spectrum != 0) or back; the steps launched by
// pstd_internal_launch_steps expect the spectrum form.  Adds the kernel count.
int pstd_internal_convert_velocity(pstd_plan_t* P, float* const* u, int to_spectrum, int64_t* launches);
// GEMM of the tensor-core split form: pstd_nn_gemm_tf32 with both operands
// split into TF32 hi + lo parts (B's lo part from B_lo, same strides as B).
int pstd_internal_tc_gemm_split(const pstd_gemm_desc* d, const float* B_lo, int* status, cudaStream_t st);
// The plan's stream.
cudaStream_t pstd_internal_stream(const pstd_plan_t* P);
// First stored pressure node per axis (0 or 1) and the pressure shape.
void pstd_internal_layout(const pstd_plan_t* P, int lo[3], int64_t shape[3]);
// Record a CUDA error text for pstd_last_cuda_error().
int pstd_internal_cuda_fail(cudaError_t e, const char* what);

// A batch of plans as one cooperative kernel per run (pstd_batch_set_persistent).
struct pstd_batch_persist_s;
// Which cooperative kernel the plans allow: 1 the register-FFT passes (every
// axis of every member on one register schedule; the velocities are in their
// spectrum form around the run, as for pstd_internal_launch_steps), 2 the
// generic CTA program on every axis (velocities as stored), 0 none (a
// dense-operator form).
int pstd_internal_batch_persist_kind(pstd_plan_t* const* plans, int n);
// Launch `nsteps` steps of every member (fields p[m], u[3 m + a]) as one
// cooperative kernel on stream st; *state (created on first use) holds the
// device copies of the passes and the grid barrier.  spin_limit: polls before
// a wait gives up (0: default); withhold: extra arrivals the barrier waits
// for (tests of the bounded wait).
int pstd_internal_batch_persist_run(pstd_batch_persist_s** state, pstd_plan_t* const* plans, int n, float* const* p,
                                    float* const* u, int64_t nsteps, long long spin_limit, unsigned withhold,
                                    cudaStream_t st);
// PSTD_ETIMEOUT once if a wait of the last cooperative run gave up (the
// caller has synchronised), else PSTD_OK.
int pstd_internal_batch_persist_status(pstd_batch_persist_s* state);
void pstd_internal_batch_persist_free(pstd_batch_persist_s* state);

// Per-operator-kind hooks used by the march driver (ops.cu).
#pragma once

#include "rsv_internal.h"

namespace rsv {

struct MarchTile {
  int64_t n0;        // first step of the tile
  int steps;         // steps in the tile
  int64_t n_forced;  // forcing is on for steps < n_forced
  int y_first;       // tile steps s >= y_first store their starting state in Y
  int kg;            // vectors in the current group
  bool adjoint;      // march with A^H
};

rsv_status build_gl1d(rsv_operator op, const rsv_operator_desc* d);
rsv_status build_dense(rsv_operator op, const rsv_operator_desc* d);
rsv_status build_adr2d(rsv_operator op, const rsv_operator_desc* d);
rsv_status build_adv3d(rsv_operator op, const rsv_operator_desc* d);
rsv_status upload(rsv_operator op, const void* host, size_t bytes, void** dst);

int default_tile_steps(rsv_operator op);
size_t stage_scratch_bytes(rsv_operator op, int kg);

// Number of kernels one march_tile call launches (for the launch accounting).
int march_tile_kernels(rsv_operator op, int steps, int kg);

// S RK4 steps of the operator's stage kernel(s) on the state block (kg vectors).
template <typename R>
cudaError_t march_tile(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y, double* norms);

// Coefficients the synthesis reads for one vector group: the input block itself
// (stage-based kinds) or a per-march transform of it (dense kind).  Sets
// *coef / *coef_stride / *n_tau_per_step.
template <typename R>
rsv_status prepare_coefficients(rsv_operator op, const void* fhat, int64_t f_stride, int kg, bool adjoint,
                                const void** coef, int64_t* coef_stride, int* synth_stride);

// Kind-specific work when the frequency grid (and so the step h) changes.
rsv_status on_frequencies(rsv_operator op);

// Sets the flag if the state block holds a NaN / Inf (kinds without an in-kernel norm monitor).
cudaError_t check_finite(rsv_operator op, const void* state, int64_t count, bool real_state);
cudaError_t state_sq_norms(rsv_operator op, int kg, int64_t n_end, double* d_out);
// Per-instance squared norms of vector 0 of the state after step n_end; the decay probe's initial state.
cudaError_t instance_sq_norms(rsv_operator op, int64_t n_end, double* d_out);
cudaError_t probe_initial_state(rsv_operator op, uint64_t seed);

// dense kind (dense_kernels.cu)
rsv_status dense_on_frequencies(rsv_operator op);
template <typename R>
cudaError_t dense_prepare(rsv_operator op, const void* fhat, int64_t f_stride, int kg, bool adjoint, void* out,
                          void* tmp);
template <typename R>
cudaError_t dense_step(rsv_operator op, int kg, bool adjoint, const void* uin, void* uout, const void* F, void* Y);
template <typename R>
cudaError_t dense_apply(rsv_operator op, const void* x, int k, bool adjoint, void* y);

// tensor-core dense step (dense_tc.cu)
bool dense_tc_supported(rsv_operator op, int kg);
size_t dense_tc_scratch_bytes(rsv_operator op);
rsv_status dense_tc_prepare(rsv_operator op, const void* d64_direct);
cudaError_t dense_tc_step(rsv_operator op, int kg, bool adjoint, int64_t step, const void* uin, void* uout,
                          const void* F, void* Y, void* xbuf);
size_t dense_tc_chain_x_bytes(rsv_operator op);
cudaError_t dense_tc_march_tile(rsv_operator op, int kg, bool adjoint, int64_t n0, int steps, int64_t n_forced,
                                int y_first, void* state, const void* F, void* Y, void* xbuf);

// structured-grid kinds (stencil_kernels.cu)
size_t stencil_scratch_bytes(rsv_operator op, int kg);
// whether FP32 marches of the 2-D / 3-D kind use the stage-pair kernels (environment switches)
bool adr2d_pairs_enabled();
bool adv3d_pairs_enabled();
template <typename R>
cudaError_t stencil_march_tile(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y);
template <typename R>
cudaError_t stencil_apply(rsv_operator op, const void* x, int k, bool adjoint, void* y);

// y = A x or A^H x for k vectors.
template <typename R>
cudaError_t apply_op(rsv_operator op, const void* x, int k, bool adjoint, void* y);

}  // namespace rsv

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
int march_group_size(rsv_operator op, int k, int S);
size_t stage_scratch_bytes(rsv_operator op, int kg);

// S RK4 steps of the operator's stage kernel(s) on the state block (kg vectors).
template <typename R>
cudaError_t march_tile(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y, double* norms);

// y = A x or A^H x for k vectors.
template <typename R>
cudaError_t apply_op(rsv_operator op, const void* x, int k, bool adjoint, void* y);

}  // namespace rsv

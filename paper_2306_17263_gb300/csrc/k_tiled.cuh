// Tiled FP32_REFINED kernels (k_tiled.cu): curl tile + solve tile per half-step.
#pragma once

#include <string>

#include "ms_internal.h"

namespace ms {

constexpr int kTiledKMax = 12;       // largest Pade band half-width the tiles hold
constexpr int kTiledMaxSweeps = 6;   // largest Richardson sweep count (halo = sweeps - 1)

// Coefficients of the FP32 step of a grid (k_mixed.cu): 12 beta, 6 c1 h^2, the Richardson
// relaxation, the increment scales 12 Z / r and 12 / (r Z), all split hi + lo; S sweeps.
struct MixedConsts {
  float cb_hi, cb_lo, d_hi, d_lo, omega, sE_hi, sE_lo, sH_hi, sH_lo;
  int S;
};
MixedConsts mixed_consts(const ms_grid* g);

int tiled_configure();
size_t tiled_curl_smem();
size_t tiled_solve_smem();
// step 0: b0 = Step 1 right-hand side on E_z; step 1: b0, b1 = Step 2 right-hand sides on H_x, H_y.
void tiled_curl(ms_grid* g, int step, float cb_hi, float cb_lo, float* b0, float* b1);
// Step 2 right-hand sides from an already filtered E_z-shaped float-float field (hi, lo).
void tiled_curl_unfiltered(ms_grid* g, const float* hi, const float* lo, float* b0, float* b1);
// S sweeps of 6 h^2 P1 x = b and the float-float update (hi, lo) += (s_hi + s_lo) x for 1 or 2 fields.
void tiled_solve(ms_grid* g, int nfields, const int* fields, const float* const* b, int S, float d_hi, float d_lo,
                 float omega, float s_hi, float s_lo);

// One launch per kernel for many cavities: per-cavity arguments and (cavity, tile) work lists.
struct CurlArgs;
struct SolveArgs;
struct TiledBatch {
  CurlArgs* d_curl = nullptr;    // [Step 1 args of every cavity][Step 2 args of every cavity]
  SolveArgs* d_solve = nullptr;  // [E solve args][H solve args]
  int* d_work = nullptr;         // curl (cavity, tile) pairs, E (cavity, slot, tile), H (cavity, slot, tile)
  int count = 0, n_curl = 0, n_solveE = 0, n_solveH = 0;
  size_t off_curl = 0, off_solveE = 0, off_solveH = 0;
};
// order: 0 cavity by cavity (row-major tiles), 1 the boundary-ring tiles of every cavity first,
// 2 largest cavities first.  persistent: launch only as many blocks as are resident at once, each
// striding over the work list.
int tiled_batch_build(ms_grid* const* cav, int count, int order, TiledBatch* tb, std::string* err);
void tiled_batch_step(const TiledBatch& tb, cudaStream_t st, int persistent);
void tiled_batch_free(TiledBatch* tb);

}  // namespace ms

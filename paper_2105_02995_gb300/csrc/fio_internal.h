// fio_internal.h -- operator object shared by the translation units of libfio (not installed).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fio.h"

namespace fio {

struct dfc;  // double-float complex (fio_kernels.cuh)

struct Stage {
  uint32_t kind, nblk, R, C;
  int64_t in_len, out_len;
  uint64_t offM, offIn, offOut;
  uint32_t level, role;
  const double2* M64 = nullptr;  // device, complex128 blocks (inside the arena)
  const float2* M32 = nullptr;   // device, complex64 copy (inside arena32)
  const dfc* Mdf = nullptr;      // device, double-float copy (inside arena_df)
  const int* in = nullptr;       // device
  const int* out = nullptr;      // device
  long long launch_rows;
  // per block: valid rows / columns (the padded tail of a block is never touched), and the CTA
  // work lists of 64-row tiles for the forward (over rows) and adjoint (over columns) directions
  const int2* dims = nullptr;      // device, nblk x (rows, cols)
  const int2* tiles_fwd = nullptr;  // device, (block, tile) pairs
  const int2* tiles_adj = nullptr;
  int ntiles_fwd = 0, ntiles_adj = 0;
  int maxcols[2] = {0, 0};  // longest valid gather list of a block: forward (cols), adjoint (rows)
  // tensor-core copies (FIO_MASK_TC): block-transposed complex64 (C x R per block), bf16 in both
  // orientations with row strides padded to a multiple of 4; 128-row tile lists
  const float2* M32t = nullptr;
  const __nv_bfloat162* Mbf = nullptr;
  const __nv_bfloat162* Mbft = nullptr;
  int ldbf = 0, ldbft = 0;
  const int2* t128_fwd = nullptr;
  const int2* t128_adj = nullptr;
  int n128_fwd = 0, n128_adj = 0;
  // kernel variant chosen by fio_autotune per [arithmetic: c128, c64, double-float, TF32, BF16,
  // split TF32][direction: forward, adjoint][right-hand-side bucket]; 0 = the built-in choice
  // (see fio_capi.cu)
  int8_t var[6][2][5] = {};
  // TMA tensor maps of the tensor-core A operands per [direction: forward (M32 / Mbf), adjoint
  // (M32t / Mbft)][element: FP32, BF16]; tma_ok marks the maps that encoded (16-byte aligned
  // rows and base)
  CUtensorMap tmap[2][2];
  bool tma_ok[2][2] = {};
  // work units of the TMA kernel per [direction][at most 1, 2, 4 row tiles per unit]: (block,
  // first 128-row tile, tiles, 0), largest first
  const int4* units[2][3] = {};
  int nunits[2][3] = {};
};

}  // namespace fio

struct fio_op_s {
  int d = 0;
  int64_t n = 0, N = 0;
  int n_bf = 0, n_hif = 0, n_root = 0;
  unsigned mask = 0;
  int64_t max_len = 0;            // longest vector between two stages (>= N)
  std::vector<fio::Stage> st;     // butterfly stages, HIF stages, root
  void* arena = nullptr;          // device copy of the packed buffer
  size_t arena_bytes = 0;
  void* arena32 = nullptr;        // complex64 copies of every stage's blocks
  size_t arena32_bytes = 0;
  void* scratch = nullptr;        // 5 work arrays of max_len x b (grown on demand)
  size_t scratch_bytes = 0;
  void* arena_tc = nullptr;       // tensor-core copies of every stage's blocks
  size_t arena_tc_bytes = 0;
  void* arena_df = nullptr;       // double-float copies of every stage's blocks
  size_t arena_df_bytes = 0;
  void* meta = nullptr;           // per-block dims and tile lists of every stage
  size_t meta_bytes = 0;
  void* units = nullptr;          // work-unit lists of the TMA kernel (every stage)
  size_t units_bytes = 0;
  void* solver = nullptr;         // solver work arrays (fio_solve.cu)
  size_t solver_bytes = 0;
};

// precisions whose stage products may run on the tensor cores (complex64 vectors)
inline bool is_tc_precision(int p) { return p == FIO_PTF32 || p == FIO_PBF16 || p == FIO_PTF32X3; }

// scratch work arrays (5 of max_len x b elements of `elem` bytes); grows with a stream sync
int fio_scratch(fio_op op, int b, size_t elem, cudaStream_t s, void** bufs);
// which: 0 K-dot, 1 K-dot*, 2 G-dot, 3 G-dot K-dot*; x, y column-major with leading dimension ld
int fio_apply_internal(fio_op op, int which, const void* x, void* y, int64_t ld, int b, int prec,
                       cudaStream_t s);
void fio_solver_free(fio_op op);
// 1 when a tensor-core kernel's bounded wait gave up since the last call (and clear the flag),
// 0 otherwise, -1 on a CUDA error
int fio_tc_timeout_reset();

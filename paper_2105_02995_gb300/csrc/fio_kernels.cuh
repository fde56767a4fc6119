// fio_kernels.cuh -- sm_103a kernels applying one packed factor stage to a batch of vectors.
//
// Every factor of K-dot, K-dot* and G-dot (paper sections 2 and 4) is a list of small dense
// complex blocks M_b with a gather list (which vector rows a block reads) and a scatter list
// (which rows it writes).  One launch applies all blocks of a stage:
//     forward  y[out_b[r]] = sum_c M_b[r][c] x[in_b[c]]
//     adjoint  y[in_b[c]]  = sum_r conj(M_b[r][c]) x[out_b[r]]
// Index -1 marks padding (reads zero, writes nothing).  Vectors are addressed as
// x[row * rs + rhs * cs], so one kernel serves the caller's column-major arrays (rs = 1,
// cs = ld) and the internal row-major work arrays (rs = b, cs = 1, one row's right-hand sides
// contiguous).
//
// Two kernel shapes:
//   k_stage_mm  b >= 5: a CTA owns one block, one tile of RT output rows and one tile of BT
//               right-hand sides; it streams the block's columns in chunks of CK through shared
//               memory (M chunk stored column-chunk-major, the gathered x chunk row-major) and
//               keeps a TR x TB register tile of complex accumulators per thread.  Each factor
//               entry is read from HBM once per right-hand-side tile.
//   k_stage_mv  b <= 4: the factor is used at most 4 times, so the kernel is a streaming matvec:
//               forward one warp per block row (lanes along the row, coalesced), adjoint one
//               thread per block column (rows walked in order, coalesced).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fio {

__device__ __forceinline__ double2 cmac(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename V>
struct StageArgs {
  const V* M;        // nblk x R x C, row-major per block
  const int* in;     // nblk x C
  const int* out;    // nblk x R
  int nblk, R, C;
  const V* x;
  long long xrs, xcs;
  V* y;
  long long yrs, ycs;
  int b;
  int ntiles;        // output-row tiles per block (when tiles == nullptr)
  const int2* dims;  // per block (valid rows, valid cols), or nullptr: the padded R x C
  const int2* tiles; // per CTA (block, 64-row tile), or nullptr: blockIdx.x = blk * ntiles + tile
  int ntiles_list;   // length of `tiles`
};

// block, row tile and valid extent of the CTA; rows/cols are in the direction of the product
template <typename V, bool ADJ>
__device__ __forceinline__ void cta_work(const StageArgs<V>& a, int& blk, int& tile, int& Rb, int& Cb) {
  if (a.tiles) {
    const int2 t = a.tiles[blockIdx.x];
    blk = t.x;
    tile = t.y;
  } else {
    blk = blockIdx.x / a.ntiles;
    tile = blockIdx.x - blk * a.ntiles;
  }
  if (a.dims) {
    const int2 d = a.dims[blk];
    Rb = d.x;
    Cb = d.y;
  } else {
    Rb = a.R;
    Cb = a.C;
  }
}

template <typename V, bool ADJ, int TX, int TB, int TR, int CK>
__global__ void __launch_bounds__(256) k_stage_mm(StageArgs<V> a) {
  constexpr int TY = 256 / TX;
  constexpr int RT = TY * TR;
  constexpr int BT = TX * TB;
  __shared__ V sM[CK][RT + 1];
  __shared__ V sX[CK][BT];

  int blk, tile, Rb, Cb;
  cta_work<V, ADJ>(a, blk, tile, Rb, Cb);
  const int j0 = blockIdx.y * BT;
  const int nrows = ADJ ? Cb : Rb;
  const int ncols = ADJ ? Rb : Cb;
  const V* M = a.M + (size_t)blk * a.R * a.C;
  const int* rowidx = ADJ ? a.in + (size_t)blk * a.C : a.out + (size_t)blk * a.R;
  const int* colidx = ADJ ? a.out + (size_t)blk * a.R : a.in + (size_t)blk * a.C;
  const int r0 = tile * RT;
  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;

  V acc[TR][TB];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int k = 0; k < TB; ++k) acc[i][k] = czero<V>();

  for (int c0 = 0; c0 < ncols; c0 += CK) {
    // op(M)[r0 + rr][c0 + cc] -> sM[cc][rr]
    for (int e = tid; e < RT * CK; e += 256) {
      int rr, cc;
      V v = czero<V>();
      if (!ADJ) {
        rr = e / CK;
        cc = e - rr * CK;
        const int r = r0 + rr, c = c0 + cc;
        if (r < nrows && c < ncols) v = M[(size_t)r * a.C + c];
      } else {
        cc = e / RT;
        rr = e - cc * RT;
        const int r = r0 + rr, c = c0 + cc;  // op(M)(r, c) = conj(M[c][r])
        if (r < nrows && c < ncols) v = cconj(M[(size_t)c * a.C + r]);
      }
      sM[cc][rr] = v;
    }
    for (int e = tid; e < CK * BT; e += 256) {
      const int cc = e / BT;
      const int jj = e - cc * BT;
      const int c = c0 + cc, j = j0 + jj;
      V v = czero<V>();
      if (c < ncols && j < a.b) {
        const int idx = colidx[c];
        if (idx >= 0) v = a.x[(long long)idx * a.xrs + (long long)j * a.xcs];
      }
      sX[cc][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < CK; ++cc) {
      V m[TR], xv[TB];
#pragma unroll
      for (int i = 0; i < TR; ++i) m[i] = sM[cc][ty + TY * i];
#pragma unroll
      for (int k = 0; k < TB; ++k) xv[k] = sX[cc][tx + TX * k];
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int k = 0; k < TB; ++k) acc[i][k] = cmac(acc[i][k], m[i], xv[k]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = r0 + ty + TY * i;
    if (r >= nrows) continue;
    const int idx = rowidx[r];
    if (idx < 0) continue;
#pragma unroll
    for (int k = 0; k < TB; ++k) {
      const int j = j0 + tx + TX * k;
      if (j < a.b) a.y[(long long)idx * a.yrs + (long long)j * a.ycs] = acc[i][k];
    }
  }
}

// ---- pipelined variant: 16-byte cp.async copies, two shared-memory buffers --------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Same contract as k_stage_mm, for the internal row-major vectors (xrs = b, xcs = 1) with every
// copied row 16-byte aligned (C * sizeof(V) and b * sizeof(V) multiples of 16).  Chunk k+1 of the
// block's columns (its M tile and its gathered x rows) is in flight while chunk k is multiplied;
// out-of-range and padding copies are zero-filled (source size 0).  Dynamic shared memory:
// 2 * (MROWS * MLD + CK * BT) * sizeof(V).
template <typename V, bool ADJ, int TX, int TB, int TR, int CK>
struct PipeShape {
  static constexpr int TY = 256 / TX, RT = TY * TR, BT = TX * TB;
  static constexpr int VPC = 16 / (int)sizeof(V);  // complex values per 16-byte copy
  static constexpr int MROWS = ADJ ? CK : RT, MCOLS = ADJ ? RT : CK, MLD = MCOLS + VPC;
  static constexpr int SMEM = 2 * (MROWS * MLD + CK * BT) * (int)sizeof(V);
};

template <typename V, bool ADJ, int TX, int TB, int TR, int CK>
__global__ void __launch_bounds__(256) k_stage_mm_pipe(StageArgs<V> a) {
  using S = PipeShape<V, ADJ, TX, TB, TR, CK>;
  constexpr int TY = S::TY, RT = S::RT, BT = S::BT, VPC = S::VPC;
  constexpr int MROWS = S::MROWS, MCOLS = S::MCOLS, MLD = S::MLD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sM = reinterpret_cast<V*>(smem_raw);
  V* sX = sM + 2 * MROWS * MLD;

  int blk, tile, Rb, Cb;
  cta_work<V, ADJ>(a, blk, tile, Rb, Cb);
  const int j0 = blockIdx.y * BT;
  const int nrows = ADJ ? Cb : Rb;
  const int ncols = ADJ ? Rb : Cb;
  const V* M = a.M + (size_t)blk * a.R * a.C;
  const int* rowidx = ADJ ? a.in + (size_t)blk * a.C : a.out + (size_t)blk * a.R;
  const int* colidx = ADJ ? a.out + (size_t)blk * a.R : a.in + (size_t)blk * a.C;
  const int r0 = tile * RT;
  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;

  auto load = [&](int buf, int c0) {
    V* dM = sM + buf * MROWS * MLD;
    constexpr int CPR = MCOLS / VPC;
    for (int e = tid; e < MROWS * CPR; e += 256) {
      const int mr = e / CPR;
      const int mc = (e - mr * CPR) * VPC;
      const int grow = (ADJ ? c0 : r0) + mr;  // row of M
      const int gcol = (ADJ ? r0 : c0) + mc;  // column of M (a 16-byte chunk may end in the
                                              // zero padding of the stored row, never beyond it)
      const bool ok = grow < Rb && gcol < Cb;
      cp_async16(dM + mr * MLD + mc, ok ? (const void*)(M + (size_t)grow * a.C + gcol) : (const void*)M,
                 ok ? 16 : 0);
    }
    V* dX = sX + buf * CK * BT;
    constexpr int CPX = BT / VPC;
    for (int e = tid; e < CK * CPX; e += 256) {
      const int cc = e / CPX;
      const int jj = (e - cc * CPX) * VPC;
      const int c = c0 + cc, j = j0 + jj;
      const int idx = c < ncols ? colidx[c] : -1;
      const bool ok = idx >= 0 && j < a.b;
      cp_async16(dX + cc * BT + jj, ok ? (const void*)(a.x + (long long)idx * a.xrs + j) : (const void*)a.x,
                 ok ? 16 : 0);
    }
    cp_async_commit();
  };

  V acc[TR][TB];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int k = 0; k < TB; ++k) acc[i][k] = czero<V>();

  const int nchunks = (ncols + CK - 1) / CK;
  load(0, 0);
  for (int k = 0; k < nchunks; ++k) {
    if (k + 1 < nchunks) {
      load((k + 1) & 1, (k + 1) * CK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const V* tM = sM + (k & 1) * MROWS * MLD;
    const V* tX = sX + (k & 1) * CK * BT;
#pragma unroll 8
    for (int cc = 0; cc < CK; ++cc) {
      V m[TR], xv[TB];
#pragma unroll
      for (int i = 0; i < TR; ++i)
        m[i] = ADJ ? cconj(tM[cc * MLD + ty + TY * i]) : tM[(ty + TY * i) * MLD + cc];
#pragma unroll
      for (int q = 0; q < TB; ++q) xv[q] = tX[cc * BT + tx + TX * q];
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int q = 0; q < TB; ++q) acc[i][q] = cmac(acc[i][q], m[i], xv[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = r0 + ty + TY * i;
    if (r >= nrows) continue;
    const int idx = rowidx[r];
    if (idx < 0) continue;
#pragma unroll
    for (int q = 0; q < TB; ++q) {
      const int j = j0 + tx + TX * q;
      if (j < a.b) a.y[(long long)idx * a.yrs + (long long)j * a.ycs] = acc[i][q];
    }
  }
}

// forward streaming matvec: one warp per block row, b <= 4
template <typename V>
__global__ void __launch_bounds__(256) k_stage_mv_fwd(StageArgs<V> a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.nblk * a.R;
  if (warp >= total) return;
  const int blk = warp / a.R;
  const int r = warp - blk * a.R;
  const int Rb = a.dims ? a.dims[blk].x : a.R;
  const int Cb = a.dims ? a.dims[blk].y : a.C;
  if (r >= Rb) return;
  const int oidx = a.out[(size_t)blk * a.R + r];
  if (oidx < 0) return;
  const V* Mr = a.M + ((size_t)blk * a.R + r) * a.C;
  const int* in = a.in + (size_t)blk * a.C;
  V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
  for (int c = lane; c < Cb; c += 32) {
    const int ic = in[c];
    if (ic < 0) continue;
    const V m = Mr[c];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < a.b) acc[j] = cmac(acc[j], m, a.x[(long long)ic * a.xrs + (long long)j * a.xcs]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j >= a.b) break;
    V v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) a.y[(long long)oidx * a.yrs + (long long)j * a.ycs] = v;
  }
}

// adjoint streaming matvec: one thread per block column, b <= 4
template <typename V>
__global__ void __launch_bounds__(256) k_stage_mv_adj(StageArgs<V> a) {
  const int blk = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int Rb = a.dims ? a.dims[blk].x : a.R;
  const int Cb = a.dims ? a.dims[blk].y : a.C;
  if (c >= Cb) return;
  const int ic = a.in[(size_t)blk * a.C + c];
  if (ic < 0) return;
  const V* M = a.M + (size_t)blk * a.R * a.C + c;
  const int* out = a.out + (size_t)blk * a.R;
  V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
  for (int r = 0; r < Rb; ++r) {
    const int orow = out[r];
    if (orow < 0) continue;
    const V m = cconj(M[(size_t)r * a.C]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < a.b) acc[j] = cmac(acc[j], m, a.x[(long long)orow * a.xrs + (long long)j * a.xcs]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j < a.b) a.y[(long long)ic * a.yrs + (long long)j * a.ycs] = acc[j];
}

// INPLACE stages compute into a scratch vector S (same row numbering) and then copy the touched
// rows back into the work vector W; blocks own disjoint rows, so no block reads a row another
// block has already overwritten.
template <typename V>
__global__ void k_scatter_back(const int* idx, long long nidx, const V* S, V* W, int b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nidx * b) return;
  const long long k = t / b;
  const int j = (int)(t - k * b);
  const int row = idx[k];
  if (row < 0) return;
  W[(long long)row * b + j] = S[(long long)row * b + j];
}

// column-major (ld) <-> row-major (b) layout changes of an N x b array, 32 x 32 smem tiles
template <typename V>
__global__ void k_col_to_row(const V* X, long long ld, V* W, long long N, int b) {
  __shared__ V t[32][33];
  const long long i0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long i = i0 + threadIdx.x;
    const int j = j0 + k;
    if (i < N && j < b) t[k][threadIdx.x] = X[i + (long long)j * ld];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long i = i0 + k;
    const int j = j0 + threadIdx.x;
    if (i < N && j < b) W[i * b + j] = t[threadIdx.x][k];
  }
}

template <typename V>
__global__ void k_row_to_col(const V* W, V* Y, long long ld, long long N, int b) {
  __shared__ V t[32][33];
  const long long i0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long i = i0 + k;
    const int j = j0 + threadIdx.x;
    if (i < N && j < b) t[k][threadIdx.x] = W[i * b + j];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long i = i0 + threadIdx.x;
    const int j = j0 + k;
    if (i < N && j < b) Y[i + (long long)j * ld] = t[threadIdx.x][k];
  }
}

__global__ void k_cast_c128_c64(const double2* a, float2* b, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

}  // namespace fio

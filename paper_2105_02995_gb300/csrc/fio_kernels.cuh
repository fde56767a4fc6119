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
//   k_stage_vec b <= 4: the factor is used at most 4 times, so the kernel streams it once,
//               coalesced, with the tile's gathered inputs in shared memory (forward: a warp
//               per row; adjoint: threads along the columns).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
// acc += conj(a) * b, with the conjugation folded into the FMAs' operand signs (the same
// operations, in the same order, as cmac(acc, cconj(a), b))
__device__ __forceinline__ double2 cmacc(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cmacc(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// ---- double-float complex: FP64-class accuracy from FP32 arithmetic -------------------------
// A value is (rh + rl) + i (ih + il) with |rl| <= ulp(rh) / 2 (the "double-float" format of
// Dekker, 1971: two non-overlapping floats, 48-bit significand).  GB300's FP64 pipes are a small
// fraction of its FP32 rate, so the FP64-accuracy residual of iterative refinement runs in this
// format.  Products are accumulated with the compensated dot product of Ogita, Rump and Oishi
// (2005, "Dot2"): each real product a*b of two double-floats is split exactly into
// ph + pe (TwoProduct by FMA, plus the cross terms ah*bl + al*bh), ph is added to the running sum
// s by Knuth's TwoSum (exact error e), and the errors e + pe collect in a compensation c; the
// result is (s, c) renormalised.  Its error is that of a sum in twice the working precision plus
// one rounding to double-float.  Arithmetic uses __fmul_rn / __fadd_rn / __fsub_rn so that no
// multiply is contracted into an FMA, which would break the error-free transformations.
struct __align__(16) dfc {
  float rh, ih, rl, il;
};
// accumulator in the same four floats: (s_re, s_im, c_re, c_im) until cfin renormalises it
__device__ __forceinline__ void dot2_step(float& s, float& c, float ah, float al, float bh, float bl) {
  const float ph = __fmul_rn(ah, bh);
  float pe = fmaf(ah, bh, -ph);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  const float t = __fadd_rn(s, ph);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(ph, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, pe));
}
__device__ __forceinline__ dfc cmac(dfc acc, dfc a, dfc b) {
  // re += a.re b.re - a.im b.im ; im += a.re b.im + a.im b.re
  dot2_step(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  dot2_step(acc.rh, acc.rl, a.ih, a.il, -b.ih, -b.il);
  dot2_step(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  dot2_step(acc.ih, acc.il, a.ih, a.il, b.rh, b.rl);
  return acc;
}
__device__ __forceinline__ dfc cconj(dfc a) { return dfc{a.rh, -a.ih, a.rl, -a.il}; }
__device__ __forceinline__ dfc cmacc(dfc acc, dfc a, dfc b) { return cmac(acc, cconj(a), b); }
template <> __device__ __forceinline__ dfc czero<dfc>() { return dfc{0.f, 0.f, 0.f, 0.f}; }
// (s, c) -> double-float (hi, lo) with hi = fl(s + c) (Fast2Sum: |c| is below ulp-scale of |s|)
__device__ __forceinline__ void df_norm(float s, float c, float& hi, float& lo) {
  hi = __fadd_rn(s, c);
  lo = __fsub_rn(c, __fsub_rn(hi, s));
}
// sum of two accumulators (s1, c1) + (s2, c2): TwoSum of the leading parts, errors to c
__device__ __forceinline__ void df_acc_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(c2, e));
}

// value stored from an accumulator (identity but for the double-float renormalisation)
__device__ __forceinline__ double2 cfin(double2 v) { return v; }
__device__ __forceinline__ float2 cfin(float2 v) { return v; }
__device__ __forceinline__ dfc cfin(dfc v) {
  dfc o;
  df_norm(v.rh, v.rl, o.rh, o.rl);
  df_norm(v.ih, v.il, o.ih, o.il);
  return o;
}
// a += b for accumulators
__device__ __forceinline__ void cacc_add(double2& a, double2 b) {
  a.x += b.x;
  a.y += b.y;
}
__device__ __forceinline__ void cacc_add(float2& a, float2 b) {
  a.x += b.x;
  a.y += b.y;
}
__device__ __forceinline__ void cacc_add(dfc& a, dfc b) {
  df_acc_add(a.rh, a.rl, b.rh, b.rl);
  df_acc_add(a.ih, a.il, b.ih, b.il);
}
// every member of a value exchanged with lane (lane ^ o)
__device__ __forceinline__ void shfl_xor_all(double2& v, int o) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
}
__device__ __forceinline__ void shfl_xor_all(float2& v, int o) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
}
__device__ __forceinline__ void shfl_xor_all(dfc& v, int o) {
  v.rh = __shfl_xor_sync(0xffffffffu, v.rh, o);
  v.ih = __shfl_xor_sync(0xffffffffu, v.ih, o);
  v.rl = __shfl_xor_sync(0xffffffffu, v.rl, o);
  v.il = __shfl_xor_sync(0xffffffffu, v.il, o);
}

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
  const int2* tiles128;  // per CTA (block, 128-row tile): the work list of 128-row tiles
  int ntiles128;
  // split over the block's columns (k_stage_mm_vt, in-place stages): blockIdx.z is the slice;
  // slice ks of row r of block blk goes to part[(ks * prow + blk * rows + r) * b + j], rows the
  // block's rows in the product's direction (summed by k_partial_reduce); part == nullptr: none
  int ksplit = 1;
  V* part = nullptr;
  long long prow = 0;
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
      if (j < a.b) a.y[(long long)idx * a.yrs + (long long)j * a.ycs] = cfin(acc[i][k]);
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

// Three real products per complex product (Gauss's form of the 3M method; error analysis in
// Higham, "Stability of a method for multiplying complex matrices with three real matrix
// multiplications", 1992) for the FP64 and double-float stage products, where every multiply is
// costly (GB300's FP64 pipes; 12 FP32 operations per double-float product).  With m = a + ib and
// x = c + id:
//     p1 += a c,  p2 += b d,  p3 += (a +- b)(c + d);  forward (p1 - p2) + i ((p3 - p1) - p2),
//                                                     adjoint (p1 + p2) + i ((p3 - p1) + p2)
// The real part is the four-product method's two sums; the imaginary part is a difference of
// three sums, whose rounding errors scale with (|a| + |b|)(|c| + |d|) instead of |a||d| + |b||c|
// (at most a few times larger).  The sums a +- b and c + d are formed once per chunk in shared
// memory (a real value of the arithmetic: a double, or a double-float pair added with TwoSum).
// G3Ops<V> is the arithmetic.
template <typename V> struct G3Ops;
template <> struct G3Ops<double2> {
  using S = double;  // a sum a +- b or c + d
  using A = double;  // one of the three running sums
  static __device__ __forceinline__ A zero() { return 0.0; }
  static __device__ __forceinline__ S sum_m(double2 m, bool adj) { return adj ? __dsub_rn(m.x, m.y) : __dadd_rn(m.x, m.y); }
  static __device__ __forceinline__ S sum_x(double2 x) { return __dadd_rn(x.x, x.y); }
  static __device__ __forceinline__ void step(A& p1, A& p2, A& p3, double2 m, S sm, double2 x, S tx) {
    p1 = fma(m.x, x.x, p1);
    p2 = fma(m.y, x.y, p2);
    p3 = fma(sm, tx, p3);
  }
  static __device__ __forceinline__ double2 fin(A p1, A p2, A p3, bool adj) {
    return adj ? make_double2(__dadd_rn(p1, p2), __dadd_rn(__dsub_rn(p3, p1), p2))
               : make_double2(__dsub_rn(p1, p2), __dsub_rn(__dsub_rn(p3, p1), p2));
  }
};
// double-float a + b (Knuth's TwoSum of the leading parts, the trailing parts and the error
// added, renormalised by Fast2Sum)
__device__ __forceinline__ float2 df_add(float ah, float al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float z = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, z)), __fsub_rn(bh, z));
  const float c = __fadd_rn(e, __fadd_rn(al, bl));
  const float hi = __fadd_rn(s, c);
  return make_float2(hi, __fsub_rn(c, __fsub_rn(hi, s)));
}
template <> struct G3Ops<dfc> {
  using S = float2;  // double-float (hi, lo)
  using A = float2;  // Dot2 accumulator (s, c)
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ S sum_m(dfc m, bool adj) {
    return adj ? df_add(m.rh, m.rl, -m.ih, -m.il) : df_add(m.rh, m.rl, m.ih, m.il);
  }
  static __device__ __forceinline__ S sum_x(dfc x) { return df_add(x.rh, x.rl, x.ih, x.il); }
  static __device__ __forceinline__ void step(A& p1, A& p2, A& p3, dfc m, S sm, dfc x, S tx) {
    dot2_step(p1.x, p1.y, m.rh, m.rl, x.rh, x.rl);
    dot2_step(p2.x, p2.y, m.ih, m.il, x.ih, x.il);
    dot2_step(p3.x, p3.y, sm.x, sm.y, tx.x, tx.y);
  }
  // the accumulator form (re s, im s, re c, im c) that cfin renormalises
  static __device__ __forceinline__ dfc fin(A p1, A p2, A p3, bool adj) {
    float rs = p1.x, rc = p1.y, is = p3.x, ic = p3.y;
    df_acc_add(rs, rc, adj ? p2.x : -p2.x, adj ? p2.y : -p2.y);
    df_acc_add(is, ic, -p1.x, -p1.y);
    df_acc_add(is, ic, adj ? p2.x : -p2.x, adj ? p2.y : -p2.y);
    return dfc{rs, is, rc, ic};
  }
};

// Same contract as k_stage_mm, for the internal row-major vectors (xrs = b, xcs = 1) with every
// copied row 16-byte aligned (C * sizeof(V) and b * sizeof(V) multiples of 16).  Chunk k+1 of the
// block's columns (its M tile and its gathered x rows) is in flight while chunk k is multiplied;
// out-of-range and padding copies are zero-filled (source size 0).  Dynamic shared memory:
// 2 * (MROWS * MLD + CK * BT) * sizeof(V), and with G3 (FP64 and double-float only) the two
// planes of sums beside the tiles, 8 bytes per entry.
template <typename V, bool ADJ, int TX, int TB, int TR, int CK>
struct PipeShape {
  static constexpr int TY = 256 / TX, RT = TY * TR, BT = TX * TB;
  static constexpr int VPC = 16 / (int)sizeof(V);  // complex values per 16-byte copy
  static constexpr int MROWS = ADJ ? CK : RT, MCOLS = ADJ ? RT : CK, MLD = MCOLS + VPC;
  static constexpr int SMEM = 2 * (MROWS * MLD + CK * BT) * (int)sizeof(V);
  static constexpr int smem(bool g3) { return SMEM + (g3 ? 2 * (MROWS * MLD + CK * BT) * 8 : 0); }
};

template <typename V, bool ADJ, int TX, int TB, int TR, int CK, bool G3 = false>
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
  // G3: the three running sums of every output and the planes of sums (types of G3Ops<V>)
  using Ops = G3Ops<typename std::conditional<G3, V, double2>::type>;
  using GS = typename Ops::S;
  using GA = typename Ops::A;
  constexpr int GR = G3 ? TR : 1, GB = G3 ? TB : 1;
  GA p1[GR][GB], p2[GR][GB], p3[GR][GB];
  GS* sS = reinterpret_cast<GS*>(sX + 2 * CK * BT);  // [2][MROWS][MLD]
  GS* sT = sS + 2 * MROWS * MLD;                      // [2][CK][BT]
  if constexpr (G3) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int k = 0; k < TB; ++k) p1[i][k] = p2[i][k] = p3[i][k] = Ops::zero();
  }

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
    if constexpr (G3) {
      // the chunk's sums, once: a +- b of every factor entry, c + d of every x entry
      GS* wS = sS + (k & 1) * MROWS * MLD;
      GS* wT = sT + (k & 1) * CK * BT;
      for (int e = tid; e < MROWS * MCOLS; e += 256) {
        const int mr = e / MCOLS, mc = e - mr * MCOLS;
        wS[mr * MLD + mc] = Ops::sum_m(tM[mr * MLD + mc], ADJ);
      }
      for (int e = tid; e < CK * BT; e += 256) wT[e] = Ops::sum_x(tX[e]);
      __syncthreads();
      const GS* tS = wS;
      const GS* tT = wT;
#pragma unroll 4
      for (int cc = 0; cc < CK; ++cc) {
        V m[TR], xv[TB];
        GS sm[TR], tx3[TB];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
          const int o = ADJ ? cc * MLD + ty + TY * i : (ty + TY * i) * MLD + cc;
          m[i] = tM[o];
          sm[i] = tS[o];
        }
#pragma unroll
        for (int q = 0; q < TB; ++q) {
          xv[q] = tX[cc * BT + tx + TX * q];
          tx3[q] = tT[cc * BT + tx + TX * q];
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int q = 0; q < TB; ++q) Ops::step(p1[i][q], p2[i][q], p3[i][q], m[i], sm[i], xv[q], tx3[q]);
      }
    } else {
#pragma unroll 8
      for (int cc = 0; cc < CK; ++cc) {
        V m[TR], xv[TB];
#pragma unroll
        for (int i = 0; i < TR; ++i) m[i] = ADJ ? tM[cc * MLD + ty + TY * i] : tM[(ty + TY * i) * MLD + cc];
#pragma unroll
        for (int q = 0; q < TB; ++q) xv[q] = tX[cc * BT + tx + TX * q];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int q = 0; q < TB; ++q) acc[i][q] = ADJ ? cmacc(acc[i][q], m[i], xv[q]) : cmac(acc[i][q], m[i], xv[q]);
      }
    }
    __syncthreads();
  }
  if constexpr (G3) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int q = 0; q < TB; ++q) acc[i][q] = Ops::fin(p1[i][q], p2[i][q], p3[i][q], ADJ);
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
      if (j < a.b) a.y[(long long)idx * a.yrs + (long long)j * a.ycs] = cfin(acc[i][q]);
    }
  }
}

// ---- complex64 variant with contiguous per-thread tiles and 16-byte shared-memory reads -------
// Same contract, tiles and copies as k_stage_mm_pipe<float2, ...> (and the same summation order
// of every output: sequential over the block's columns), with NT threads and thread (tx, ty)
// owning rows ty*TR .. ty*TR+TR-1 and right-hand sides tx*TB .. tx*TB+TB-1 of the CTA tile.  The
// adjoint reads its TR conjugated factor entries of one column (contiguous in the tile) and both
// directions read their TB vector entries as float4 pairs, halving the shared-memory
// instructions per FMA; TR = 8 with 128 threads gives 16 accumulators per thread.  With 8 x 4
// thread tiles (<8,4,8> on 128 threads) a CTA covers 128 rows and 32 right-hand sides: 32
// accumulators per thread, 128 FMAs per step of the column loop against 10 shared-memory loads
// (6 in the adjoint), from the list of 128-row tiles, with chunks of 16 columns.
//
// Shared-memory layout of the 8 x 4 tiles (TX = 8: a warp holds 4 thread rows ty and 8 thread
// columns tx).  Unpadded, the 4 ty of a warp read factor entries 64 bytes apart in the adjoint
// (TR = 8 contiguous values each) or whole rows apart in the forward direction, and the 8 tx read
// vector entries 32 bytes apart: two or four accesses per shared-memory bank.  Two complex
// values of padding after every 8 factor columns (adjoint) or 8 factor rows (forward), and after
// every 4 vector entries, put every access of a warp in a bank of its own (PA, PF, PX).  The
// column indices of the next chunk's gathered rows are loaded into registers one chunk ahead, so
// the cp.async copies of a chunk never wait for an index load.  The 8 x 4 tiles are held to 128
// registers a thread by default (MINB = 4 CTAs, 16 warps, per SM); MINB = 1 lets the compiler
// use more (the adjoint then takes about 155, three CTAs per SM).
template <bool ADJ, int TX, int TB, int TR, int NT, int CK_ = 32>
struct VtShape {
  static constexpr int TY = NT / TX, RT = TY * TR, BT = TX * TB, CK = CK_;
  static constexpr int MROWS = ADJ ? CK : RT, MCOLS = ADJ ? RT : CK;
  static constexpr int PA = (ADJ && TR == 8 && TX == 8) ? 2 : 0;   // per 8 factor columns
  static constexpr int PF = (!ADJ && TR == 8 && TX == 8) ? 2 : 0;  // per 8 factor rows
  static constexpr int PX = (TB == 4 && TX == 8) ? 2 : 0;          // per 4 vector entries
  static constexpr int MLD = MCOLS + 2 + (MCOLS / 8) * PA;
  static constexpr int MTILE = MROWS * MLD + (MROWS / 8) * PF;
  static constexpr int BTP = BT + (BT / 4) * PX;
  static constexpr int XTILE = CK * BTP;
  static constexpr int SMEM = 2 * (MTILE + XTILE) * 8;
  // offset of factor entry (row mr, column mc) of a tile, and of vector entry j of chunk column cc
  static __device__ __forceinline__ int mofs(int mr, int mc) {
    return mr * MLD + (mr >> 3) * PF + mc + (mc >> 3) * PA;
  }
  static __device__ __forceinline__ int xofs(int cc, int j) { return cc * BTP + j + (j >> 2) * PX; }
};

template <bool ADJ, int TX, int TB, int TR, int NT, int CK_ = 32, int MINB = (NT == 128 && TX == 8 ? 4 : 1)>
__global__ void __launch_bounds__(NT, MINB) k_stage_mm_vt(StageArgs<float2> a) {
  using S = VtShape<ADJ, TX, TB, TR, NT, CK_>;
  constexpr int RT = S::RT, BT = S::BT, CK = S::CK;
  constexpr int MROWS = S::MROWS, MCOLS = S::MCOLS, MTILE = S::MTILE, XTILE = S::XTILE;
  static_assert(TB % 2 == 0 && TR % 2 == 0 && (RT == 64 || RT == 128), "tile shape");
  static_assert(S::PA == 0 || TR == 8, "adjoint padding groups a thread's 8 rows");
  static_assert(S::PX == 0 || TB == 4, "vector padding groups a thread's 4 right-hand sides");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sM = reinterpret_cast<float2*>(smem_raw);
  float2* sX = sM + 2 * MTILE;

  int blk, tile, Rb, Cb;
  cta_work<float2, ADJ>(a, blk, tile, Rb, Cb);
  const int j0 = blockIdx.y * BT;
  const int nrows = ADJ ? Cb : Rb;
  const int ncols = ADJ ? Rb : Cb;
  const float2* M = a.M + (size_t)blk * a.R * a.C;
  const int* rowidx = ADJ ? a.in + (size_t)blk * a.C : a.out + (size_t)blk * a.R;
  const int* colidx = ADJ ? a.out + (size_t)blk * a.R : a.in + (size_t)blk * a.C;
  const int r0 = tile * RT;
  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;

  // x pairs this thread copies per chunk, and the column indices of the next chunk's pairs
  constexpr int CPX = BT / 2;
  constexpr int NXP = (CK * CPX + NT - 1) / NT;
  int nidx[NXP];
  auto fetch_idx = [&](int c0) {
#pragma unroll
    for (int u = 0; u < NXP; ++u) {
      const int e = tid + u * NT;
      const int c = c0 + e / CPX;
      nidx[u] = (e < CK * CPX && c < ncols) ? colidx[c] : -1;
    }
  };
  auto load = [&](int buf, int c0) {
    float2* dM = sM + buf * MTILE;
    constexpr int CPR = MCOLS / 2;
    for (int e = tid; e < MROWS * CPR; e += NT) {
      const int mr = e / CPR;
      const int mc = (e - mr * CPR) * 2;
      const int grow = (ADJ ? c0 : r0) + mr;
      const int gcol = (ADJ ? r0 : c0) + mc;
      const bool ok = grow < Rb && gcol < Cb;
      cp_async16(dM + S::mofs(mr, mc), ok ? (const void*)(M + (size_t)grow * a.C + gcol) : (const void*)M,
                 ok ? 16 : 0);
    }
    float2* dX = sX + buf * XTILE;
#pragma unroll
    for (int u = 0; u < NXP; ++u) {
      const int e = tid + u * NT;
      if (e < CK * CPX) {
        const int cc = e / CPX;
        const int jj = (e - cc * CPX) * 2;
        const int j = j0 + jj;
        const int idx = nidx[u];
        const bool ok = idx >= 0 && j < a.b;
        cp_async16(dX + S::xofs(cc, jj), ok ? (const void*)(a.x + (long long)idx * a.xrs + j) : (const void*)a.x,
                   ok ? 16 : 0);
      }
    }
    cp_async_commit();
    fetch_idx(c0 + CK);
  };

  float2 acc[TR][TB];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int k = 0; k < TB; ++k) acc[i][k] = make_float2(0.f, 0.f);

  // the slice of the block's column chunks this CTA sums (all of them unless split)
  const int nch = (ncols + CK - 1) / CK;
  const int cps = (nch + a.ksplit - 1) / a.ksplit;
  const int kb = min(nch, (int)blockIdx.z * cps);
  const int nchunks = min(nch, kb + cps) - kb;
  if (nchunks > 0) {
    fetch_idx(kb * CK);
    load(0, kb * CK);
  }
  for (int k = 0; k < nchunks; ++k) {
    if (k + 1 < nchunks) {
      load((k + 1) & 1, (kb + k + 1) * CK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* tM = sM + (k & 1) * MTILE;
    const float2* tX = sX + (k & 1) * XTILE;
#pragma unroll 4
    for (int cc = 0; cc < CK; ++cc) {
      float2 m[TR], xv[TB];
      if (ADJ) {
#pragma unroll
        for (int i = 0; i < TR; i += 2) {
          const float4 v = *reinterpret_cast<const float4*>(tM + S::mofs(cc, ty * TR + i));
          m[i] = make_float2(v.x, v.y);
          m[i + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < TR; ++i) m[i] = tM[S::mofs(ty * TR + i, cc)];
      }
#pragma unroll
      for (int q = 0; q < TB; q += 2) {
        const float4 v = *reinterpret_cast<const float4*>(tX + S::xofs(cc, tx * TB + q));
        xv[q] = make_float2(v.x, v.y);
        xv[q + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int q = 0; q < TB; ++q) acc[i][q] = ADJ ? cmacc(acc[i][q], m[i], xv[q]) : cmac(acc[i][q], m[i], xv[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = r0 + ty * TR + i;
    if (r >= nrows) continue;
    const int idx = rowidx[r];
    if (idx < 0) continue;
    float2* dst = a.part ? a.part + ((long long)blockIdx.z * a.prow + (long long)blk * (ADJ ? a.C : a.R) + r) * a.b
                         : a.y + (long long)idx * a.yrs;
    const long long cs = a.part ? 1 : a.ycs;
#pragma unroll
    for (int q = 0; q < TB; ++q) {
      const int j = j0 + tx * TB + q;
      if (j < a.b) dst[(long long)j * cs] = acc[i][q];
    }
  }
}

// ---- small blocks (padded R, C <= 32, the 16-point leaf stages): one warp per block ------------
// Lane j owns right-hand side j0 + j of the CTA's 32-wide tile.  The warp copies its block (R x C
// values, coalesced) and the block's gathered input rows (ncols x 32 values, one coalesced row
// per column) into shared memory, then every lane forms each output row as the plain sum over
// the block's columns in order, with the multiply-adds of cmac / cmacc: the same operations in the
// same order as the tiled kernels (which add only zeros beyond the valid columns), so the results
// are bit-identical to theirs.  A 64- or 128-row tile would leave most of its rows idle on a
// 16 x 16 block.  Dynamic shared memory: kSmallWarps x (R C + 32 cmax) values, cmax = C forward,
// R adjoint.
constexpr int kSmallWarps = 4;
constexpr int kSmallMaxDim = 32;

template <typename V, bool ADJ>
__global__ void __launch_bounds__(32 * kSmallWarps) k_stage_small(StageArgs<V> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int blk = blockIdx.x * kSmallWarps + w;
  if (blk >= a.nblk) return;  // warp-uniform; the kernel has no CTA-wide barrier
  const int RC = a.R * a.C, cmax = ADJ ? a.R : a.C;
  V* sm = reinterpret_cast<V*>(smem_raw) + (size_t)w * (RC + 32 * cmax);
  V* sx = sm + RC;
  int Rb = a.R, Cb = a.C;
  if (a.dims) {
    const int2 d = a.dims[blk];
    Rb = d.x;
    Cb = d.y;
  }
  const int nrows = ADJ ? Cb : Rb;
  const int ncols = ADJ ? Rb : Cb;
  const V* M = a.M + (size_t)blk * RC;
  const int* rowidx = ADJ ? a.in + (size_t)blk * a.C : a.out + (size_t)blk * a.R;
  const int* colidx = ADJ ? a.out + (size_t)blk * a.R : a.in + (size_t)blk * a.C;
  for (int e = lane; e < RC; e += 32) sm[e] = M[e];
  const int j = blockIdx.y * 32 + lane;
  const bool on = j < a.b;
#pragma unroll 4
  for (int c = 0; c < ncols; ++c) {
    const int idx = colidx[c];
    sx[c * 32 + lane] = (idx >= 0 && on) ? a.x[(long long)idx * a.xrs + (long long)j * a.xcs] : czero<V>();
  }
  __syncwarp();
  for (int r = 0; r < nrows; ++r) {
    const int oidx = rowidx[r];
    if (oidx < 0) continue;
    V acc = czero<V>();
    for (int c = 0; c < ncols; ++c) {
      const V m = ADJ ? sm[c * a.C + r] : sm[r * a.C + c];
      acc = ADJ ? cmacc(acc, m, sx[c * 32 + lane]) : cmac(acc, m, sx[c * 32 + lane]);
    }
    if (on) a.y[(long long)oidx * a.yrs + (long long)j * a.ycs] = acc;
  }
}

// ---- few right-hand sides (b <= 4): one CTA per (block, 64-row tile) ------------------------
// The tile's gathered input rows (ncols x b values) are copied once into shared memory, laid out
// right-hand-side major (sX[j * ncols + c]) so that consecutive c sit in consecutive slots; the
// factor is then streamed once, coalesced, with the work split to the block's width (butterfly
// blocks can be as narrow as one 16-point leaf):
//   forward  groups of w lanes (w = 4 .. 32, about ncols / 4 rounded up to a power of two) own
//            one row each and stride along it; the row's sums are reduced within the group;
//   adjoint  the tile's T output columns (T = 4 .. 64, a power of two >= its valid columns) each
//            get 256 / T threads that take every (256 / T)-th row; the partial sums are added by
//            a tree in shared memory.
// Dynamic shared memory: max(ncols * b, ADJ ? 256 * b : 0) values.
constexpr int kVecMaxRhs = 4;

// forward rows of k_stage_vec: groups of W lanes, one row per group, B right-hand sides
template <typename V, int W, int B>
__device__ __forceinline__ void vec_rows(const StageArgs<V>& a, const V* M, const int* rowidx, const V* sX,
                                         int r0, int nrows, int ncols) {
  constexpr int PER_WARP = 32 / W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = lane & (W - 1);
  const int nr = min(64, nrows - r0);
  for (int rb = warp * PER_WARP; rb < nr; rb += 8 * PER_WARP) {  // warp-uniform trip count
    const int rr = rb + lane / W;
    const bool live = rr < nr;
    V acc[B];
#pragma unroll
    for (int j = 0; j < B; ++j) acc[j] = czero<V>();
    if (live) {
      const V* Mr = M + (size_t)(r0 + rr) * a.C;
#pragma unroll 4
      for (int c = sub; c < ncols; c += W) {
        const V m = Mr[c];
#pragma unroll
        for (int j = 0; j < B; ++j) acc[j] = cmac(acc[j], m, sX[j * ncols + c]);
      }
    }
    const int oidx = live ? rowidx[r0 + rr] : -1;
#pragma unroll
    for (int j = 0; j < B; ++j) {
      V v = acc[j];
#pragma unroll
      for (int o = W >> 1; o > 0; o >>= 1) {
        V t = v;
        shfl_xor_all(t, o);
        cacc_add(v, t);
      }
      if (sub == 0 && oidx >= 0) a.y[(long long)oidx * a.yrs + (long long)j * a.ycs] = cfin(v);
    }
  }
}

// The number of right-hand sides B (1..4) is a template parameter: every accumulator slot is
// live, so no predicated-off multiply occupies an issue slot (on GB300 an FP64 FMA slot is
// scarce).
template <typename V, bool ADJ, int B>
__global__ void __launch_bounds__(256) k_stage_vec(StageArgs<V> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sX = reinterpret_cast<V*>(smem_raw);
  int blk, tile, Rb, Cb;
  cta_work<V, ADJ>(a, blk, tile, Rb, Cb);
  const int nrows = ADJ ? Cb : Rb;
  const int ncols = ADJ ? Rb : Cb;
  const V* M = a.M + (size_t)blk * a.R * a.C;
  const int* rowidx = ADJ ? a.in + (size_t)blk * a.C : a.out + (size_t)blk * a.R;
  const int* colidx = ADJ ? a.out + (size_t)blk * a.R : a.in + (size_t)blk * a.C;
  const int r0 = tile * 64;
  const int tid = threadIdx.x;
  for (int e = tid; e < ncols * B; e += 256) {
    const int j = e / ncols, c = e - j * ncols;
    const int idx = colidx[c];
    sX[e] = idx >= 0 ? a.x[(long long)idx * a.xrs + (long long)j * a.xcs] : czero<V>();
  }
  __syncthreads();
  if (!ADJ) {
    int w = 4;
    while (w < 32 && 4 * w < ncols) w <<= 1;
    switch (w) {  // uniform per CTA; a compile-time group width keeps the row loop unrolled
      case 4: vec_rows<V, 4, B>(a, M, rowidx, sX, r0, nrows, ncols); break;
      case 8: vec_rows<V, 8, B>(a, M, rowidx, sX, r0, nrows, ncols); break;
      case 16: vec_rows<V, 16, B>(a, M, rowidx, sX, r0, nrows, ncols); break;
      default: vec_rows<V, 32, B>(a, M, rowidx, sX, r0, nrows, ncols); break;
    }
  } else {
    const int nc = min(64, nrows - r0);
    int T = 4;
    while (T < nc) T <<= 1;
    const int G = 256 / T;
    const int cl = tid & (T - 1), g = tid / T, c = r0 + cl;
    V acc[B];
#pragma unroll
    for (int j = 0; j < B; ++j) acc[j] = czero<V>();
    if (cl < nc) {
      for (int r = g; r < ncols; r += G) {
        const V m = M[(size_t)r * a.C + c];
#pragma unroll
        for (int j = 0; j < B; ++j) acc[j] = cmacc(acc[j], m, sX[j * ncols + r]);
      }
    }
    __syncthreads();  // every thread is done with sX: reuse it for the partial sums
#pragma unroll
    for (int j = 0; j < B; ++j) sX[j * 256 + tid] = acc[j];
    for (int h = G >> 1; h > 0; h >>= 1) {
      __syncthreads();
      if (g < h) {
#pragma unroll
        for (int j = 0; j < B; ++j) {
          V v = sX[j * 256 + tid];
          cacc_add(v, sX[j * 256 + tid + h * T]);
          sX[j * 256 + tid] = v;
        }
      }
    }
    __syncthreads();
    if (g == 0 && cl < nc) {
      const int oidx = rowidx[c];
      if (oidx >= 0) {
#pragma unroll
        for (int j = 0; j < B; ++j) a.y[(long long)oidx * a.yrs + (long long)j * a.ycs] = cfin(sX[j * 256 + tid]);
      }
    }
  }
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

// complex128 -> double-float: hi = fl32(v), lo = fl32(v - hi) (v - hi is exact in FP64)
__device__ __forceinline__ dfc split_df(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return dfc{rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih)};
}
__global__ void k_split_df(const double2* a, dfc* b, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = split_df(a[t]);
}
// N x b column-major complex128 (leading dimension ld) -> double-float (leading dimension N), and back
__global__ void k_c128_to_df(const double2* x, long long ld, dfc* y, long long N, int b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * b) return;
  const long long j = t / N, i = t - j * N;
  y[t] = split_df(x[j * ld + i]);
}
__global__ void k_df_to_c128(const dfc* y, long long N, double2* x, long long ld, int b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * b) return;
  const long long j = t / N, i = t - j * N;
  const dfc v = y[t];
  x[j * ld + i] = make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}

}  // namespace fio

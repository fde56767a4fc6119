// fio_tc.cuh -- tcgen05 tensor-core stage kernel (sm_103a) for batched right-hand sides.
//
// One stage block product y = op(M) x with complex M (rows x cols) and b right-hand sides is the
// real GEMM
//     [y_re y_im]-interleaved (rows x 2b)  =  A (rows x 2 cols)  *  B (2 cols x 2b)
// where A is the block's complex row data read as interleaved reals (re, im, re, im, ...) -- the
// stored factor itself, already "K-major" -- and B is built from the gathered x rows:
//     forward  (y = M x):   B[2c][2j] = xr,  B[2c+1][2j] = -xi,  B[2c][2j+1] = xi, B[2c+1][2j+1] = xr
//     adjoint  (y = M^H x, A = the block-transposed copy M^T):
//                           B[2c][2j] = xr,  B[2c+1][2j] =  xi,  B[2c][2j+1] = xi, B[2c+1][2j+1] = -xr
// so the (re, im) pair of output (r, j) lands in accumulator columns 2j, 2j+1 of row r.
//
// CTA = 128 threads, one 128-row tile of one block and up to 64 right-hand sides: accumulator
// D[128 x 2bp] fp32 in tensor memory (TMEM), operands in shared memory in the canonical K-major
// layout with 128-byte swizzle (8-row x 128-byte atoms, 1024 bytes apart).  The block's columns
// are consumed in chunks of 128 bytes of K per row (16 complex in TF32, 32 in BF16): the A tile
// and the chunk's gathered x rows arrive by 16-byte cp.async, the threads expand the x rows into
// the B tile, one elected thread issues four tcgen05.mma (K = 8 TF32 / 16 BF16 each) and commits
// them to an mbarrier; the tiles are refilled once that phase completes (waits bounded by
// %globaltimer: after kWaitNs the kernel records a timeout and stops issuing).  One operand buffer
// per CTA keeps shared memory near 30 KB so that six to seven CTAs share an SM and overlap one
// another's copies and MMAs; measured faster than two or three buffers per CTA at fewer CTAs.
// Tensor memory is allocated by warp 0 and freed on every path.
//
// Split-TF32 mode (kTcX3): FP32-accurate products on the TF32 tensor cores.  Every operand value
// v is split as v = hi + lo with hi = round-to-nearest TF32(v) and lo = TF32(v - hi) (v - hi is
// exact in FP32); the chunk's product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (twelve
// MMAs per chunk instead of four), dropping only A_lo B_lo, of relative size 2^-22.  The A tile
// is split in shared memory after it lands (hi written back in place, lo into a second tile), so
// the HBM traffic is that of the TF32 mode; B is split while it is expanded.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fio {

__device__ int g_tc_timeout;  // set when a bounded wait in k_stage_tc gave up

namespace tc {

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared memory descriptor: K-major, 128-byte swizzle, atoms of 8 rows x 128 bytes 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused: K of one MMA < 128 B)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}
// instruction descriptor: D fp32, A/B format (2 = TF32 under kind::tf32, 1 = BF16 under kind::f16),
// both K-major, N and M
__host__ __device__ constexpr uint32_t idesc(uint32_t ab_fmt, int M, int N) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// round to the nearest TF32 value (ties away from zero), returned in FP32 format
__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (BF16)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
// arrive on `bar` once every cp.async this thread issued so far has landed (counts as one arrival)
__device__ __forceinline__ void cp_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

// byte offset of (row, 16-byte chunk) in a K-major 128-byte-swizzled tile
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

}  // namespace tc

struct TcArgs {
  const void* A;      // op-matrix blocks: float2 (TF32, split TF32) or __nv_bfloat162 (BF16), row-major
  long long bstride;  // elements between blocks
  int lda;            // elements between rows
  const int* rowidx;  // output index list base (out for forward, in for adjoint), per block stride
  const int* colidx;  // input index list base
  int ldr, ldc;       // index-list strides per block (R or C of the packed stage)
  const int2* dims;   // per block (valid rows, valid cols) of the forward block
  const int2* tiles;  // per CTA (block, 128-row tile)
  const float2* x;
  long long xrs, xcs;
  float2* y;
  long long yrs, ycs;
  int b;
  int nmax;           // accumulator width N of a full right-hand-side tile (sets the smem layout)
  int stage_x;        // x rows are 16-byte aligned and contiguous: gather them with cp.async
  int ncmax;          // longest gather list of a block (sizes the shared copy of the list)
};

constexpr int kTcRows = 128;
constexpr int kTcMaxRhs = 64;  // right-hand sides per CTA (N = 128 accumulator columns)
// operand modes of k_stage_tc
constexpr int kTcTF32 = 1, kTcBF16 = 2, kTcX3 = 3;
// dynamic shared memory: A tile (16 KB) + B tile (N x 128 B) (both twice in split-TF32 mode) +
// staging of the chunk's x rows (KC rows x N/2 complex) + alignment slack, for accumulator width
// N (= 2 x right-hand sides) + the block's gather list (ncmax int32)
__host__ __device__ constexpr int tc_smem_bytes(int mode, int N, int ncmax) {
  return (mode == kTcX3 ? 2 : 1) * (16384 + N * 128) + (mode == kTcBF16 ? 32 : 16) * (N / 2) * 8 + 1024 +
         ((ncmax + 3) & ~3) * 4;
}

template <bool ADJ, int MODE>
__global__ void __launch_bounds__(128) k_stage_tc(TcArgs a) {
  using namespace tc;
  constexpr bool BF16 = MODE == kTcBF16;
  constexpr bool X3 = MODE == kTcX3;
  constexpr uint32_t TA = X3 ? 32768u : 16384u;  // bytes of the A tile(s)
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(8) uint64_t s_drain;  // after a timeout: every MMA issued has finished
  extern __shared__ __align__(16) uint8_t smem_dyn[];
  // layout: A tile (16 KB, 1024-byte aligned for the swizzle atoms; split mode: A_hi then A_lo),
  // B tile (N x 128 B; split mode: B_hi then B_lo), x staging (KC rows x nmax/2 complex), gather list
  const uint32_t base = (su32(smem_dyn) + 1023u) & ~1023u;
  uint8_t* gbase = smem_dyn + (base - su32(smem_dyn));
  const uint32_t TB = (uint32_t)a.nmax * 128;  // bytes of one B tile (a multiple of 2048)
  const uint32_t sA = base, sB = base + TA;
  uint8_t* pA = gbase;
  uint8_t* pB = gbase + TA;
  const uint32_t sX = sB + (X3 ? 2 : 1) * TB;
  const float2* pX = reinterpret_cast<const float2*>(gbase + TA + (X3 ? 2 : 1) * TB);
  int* sIdx = reinterpret_cast<int*>(gbase + TA + (X3 ? 2 : 1) * TB + (BF16 ? 32 : 16) * (a.nmax / 2) * 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int2 t = a.tiles[blockIdx.x];
  const int blk = t.x, r0 = t.y * kTcRows;
  const int2 d = a.dims[blk];
  const int nrows = ADJ ? d.y : d.x, ncols = ADJ ? d.x : d.y;
  const int j0 = blockIdx.y * kTcMaxRhs;
  const int bcta = min(kTcMaxRhs, a.b - j0);
  const int bp = (bcta + 7) & ~7;  // right-hand sides padded to 8: N = 2 bp, a multiple of 16
  const int N = 2 * bp;
  const int sld = a.nmax / 2;      // staging row length (complex)
  const uint32_t ncol_tmem = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  const int* rowidx = a.rowidx + (size_t)blk * (ADJ ? a.ldc : a.ldr);
  const int* colidx = a.colidx + (size_t)blk * (ADJ ? a.ldr : a.ldc);
  constexpr int ESZ = BF16 ? 4 : 8;  // bytes per complex entry of A
  constexpr int KC = 128 / ESZ;      // complex columns per 128-byte chunk
  constexpr int CPC = 16 / ESZ;      // complex entries per 16-byte copy
  const uint8_t* Ab = (const uint8_t*)a.A + (size_t)blk * a.bstride * ESZ;
  const uint32_t id = idesc(BF16 ? 1u : 2u, kTcRows, N);
  const int nchunks = (ncols + KC - 1) / KC;

  if (warp == 0) tmem_alloc(&s_tmem, ncol_tmem);
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    mbar_init(&s_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the block's gather list, once per CTA: the per-chunk copies then never wait on it
  for (int e = tid; e < ncols; e += 128) sIdx[e] = colidx[e];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  bool ok = true;
  for (int k = 0; k < nchunks && ok; ++k) {
    const int c0 = k * KC;
    // the previous chunk's MMAs must be done with the tiles before they are overwritten
    if (k >= 1) {
      ok = __syncthreads_and(mbar_wait(&s_bar, (uint32_t)((k - 1) & 1)) ? 1 : 0) != 0;
      fence_after();
      if (!ok) break;
    }
    // A tile: 128 rows x 128 bytes of the block, 16-byte cp.async, zero fill outside the block
    for (int e = tid; e < kTcRows * 8; e += 128) {
      const int row = e >> 3, ch = e & 7;
      const int gr = r0 + row, gc = c0 + ch * CPC;
      const bool in = gr < nrows && gc < ncols;
      const void* src = in ? (const void*)(Ab + ((size_t)gr * a.lda + gc) * ESZ) : a.A;
      cp16(sA + swz(row, ch), src, in ? 16 : 0);
    }
    if (a.stage_x) {
      // the chunk's gathered x rows (bcta complex each, contiguous): 16-byte copies into staging
      const int cpr = bcta >> 1;
      for (int e = tid; e < KC * cpr; e += 128) {
        const int c = e / cpr, q = e - c * cpr;
        const int idx = (c0 + c < ncols) ? sIdx[c0 + c] : -1;
        const void* src = idx >= 0 ? (const void*)(a.x + (long long)idx * a.xrs + j0 + 2 * q) : (const void*)a.x;
        cp16(sX + (uint32_t)((c * sld + 2 * q) * 8), src, idx >= 0 ? 16 : 0);
      }
    }
    cp_wait_all();
    __syncthreads();
    // B^T tile: rows 2j / 2j+1 = real / imaginary part of output j; K = (2c, 2c+1)
    for (int e = tid; e < KC * bp; e += 128) {
      const int c = e / bp, j = e - c * bp;
      float2 v = make_float2(0.f, 0.f);
      if (j < bcta) {
        if (a.stage_x) {
          v = pX[c * sld + j];
        } else if (c0 + c < ncols) {
          const int idx = sIdx[c0 + c];
          if (idx >= 0) v = a.x[(long long)idx * a.xrs + (long long)(j0 + j) * a.xcs];
        }
      }
      float p0, p1, q0, q1;
      if (!ADJ) {
        p0 = v.x; p1 = -v.y; q0 = v.y; q1 = v.x;
      } else {
        p0 = v.x; p1 = v.y; q0 = v.y; q1 = -v.x;
      }
      const int n0 = 2 * j, n1 = 2 * j + 1;
      if (BF16) {
        const int ch = c >> 2, off = (c & 3) << 2;
        *reinterpret_cast<__nv_bfloat162*>(pB + swz(n0, ch) + off) = __floats2bfloat162_rn(p0, p1);
        *reinterpret_cast<__nv_bfloat162*>(pB + swz(n1, ch) + off) = __floats2bfloat162_rn(q0, q1);
      } else if (X3) {
        const int ch = c >> 1, off = (c & 1) << 3;
        const float hp0 = tf32_rna(p0), hp1 = tf32_rna(p1), hq0 = tf32_rna(q0), hq1 = tf32_rna(q1);
        *reinterpret_cast<float2*>(pB + swz(n0, ch) + off) = make_float2(hp0, hp1);
        *reinterpret_cast<float2*>(pB + swz(n1, ch) + off) = make_float2(hq0, hq1);
        *reinterpret_cast<float2*>(pB + TB + swz(n0, ch) + off) =
            make_float2(tf32_rna(p0 - hp0), tf32_rna(p1 - hp1));
        *reinterpret_cast<float2*>(pB + TB + swz(n1, ch) + off) =
            make_float2(tf32_rna(q0 - hq0), tf32_rna(q1 - hq1));
      } else {
        const int ch = c >> 1, off = (c & 1) << 3;
        *reinterpret_cast<float2*>(pB + swz(n0, ch) + off) = make_float2(p0, p1);
        *reinterpret_cast<float2*>(pB + swz(n1, ch) + off) = make_float2(q0, q1);
      }
    }
    if (X3) {
      // split the A tile in place: the split is elementwise, so A_lo takes the same swizzled layout
      for (int e = tid; e < kTcRows * 8; e += 128) {
        float4* h = reinterpret_cast<float4*>(pA + 16 * e);
        const float4 v = *h;
        const float4 hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
        *h = hi;
        *reinterpret_cast<float4*>(pA + 16384 + 16 * e) =
            make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z), tf32_rna(v.w - hi.w));
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      if (X3) {
        // small terms first: the four A_lo B_hi steps of the chunk, then per step A_hi B_lo and
        // A_hi B_hi (the order of the TMA kernel, which releases the A_lo tile after its four)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          mma<false>(tmem, sdesc(sA + 16384 + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          mma<false>(tmem, sdesc(sA + 32 * q), sdesc(sB + TB + 32 * q), id, 1u);
          mma<false>(tmem, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, 1u);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          mma<BF16>(tmem, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
      }
      mma_commit(&s_bar);
    }
  }
  // drain: the last commit tracks every MMA issued before it
  if (nchunks > 0 && ok) {
    ok = __syncthreads_and(mbar_wait(&s_bar, (uint32_t)((nchunks - 1) & 1)) ? 1 : 0) != 0;
    fence_after();
  }
  cp_wait_all();
  if (!ok) {
    // a wait gave up with MMAs possibly still in flight: thread 0 (which issued all of them)
    // commits once more, and the CTA waits (bounded) for that commit before the tiles and the
    // tensor memory are released
    if (tid == 0) {
      atomicExch(&g_tc_timeout, 1);
      mma_commit(&s_drain);
    }
    __syncthreads();
    mbar_wait(&s_drain, 0);
    fence_after();
  }

  // epilogue: warp w holds accumulator rows 32w .. 32w+31 (TMEM lanes)
  const int row = r0 + warp * 32 + lane;
  const int oidx = (row < nrows) ? rowidx[row] : -1;
  for (int cb = 0; cb < N; cb += 16) {
    uint32_t r[16];
    if (nchunks > 0 && ok) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) r[q] = 0u;
    }
    if (oidx >= 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = cb / 2 + q;
        if (j < bcta)
          a.y[(long long)oidx * a.yrs + (long long)(j0 + j) * a.ycs] =
              make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncol_tmem);
}

// ---- warp-specialised ring variant ----------------------------------------------------------
// Same product and operand layout as k_stage_tc, with S chunk stages in shared memory and the
// work split by role so that copies, B expansion and MMAs of different chunks overlap inside
// one CTA (192 threads):
//   warp 4      producer: 16-byte cp.async of chunk k's A tile and gathered x rows into stage
//               k mod S, once the MMAs of chunk k - S have released it (mbarrier `empty`); the
//               copies' completion arrives on `full` (cp.async.mbarrier.arrive.noinc);
//   warps 0-3   expand the staged x rows into the B tile (split mode: also split the A tile),
//               fence the writes to the async proxy and arrive on `bready`; after the last
//               chunk they read the accumulator out of TMEM (lane quadrant = warp) and store;
//   warp 5      lane 0 issues the chunk's MMAs when `bready` completes and commits them to
//               `empty` (and, after the last chunk, to `done`).
// Every wait is bounded (kWaitNs): a role that gives up stops, the others give up in turn, the
// timeout is recorded, and the CTA still waits for its copies and MMAs before freeing TMEM.
__host__ __device__ constexpr int tc_ring_stage_bytes(int mode, int N) {
  return (((mode == kTcX3 ? 2 : 1) * (16384 + N * 128) + (mode == kTcBF16 ? 32 : 16) * (N / 2) * 8) + 1023) &
         ~1023;
}
__host__ __device__ constexpr int tc_ring_smem_bytes(int mode, int N, int ncmax, int S) {
  return S * tc_ring_stage_bytes(mode, N) + 1024 + ((ncmax + 3) & ~3) * 4;
}

template <bool ADJ, int MODE, int S>
__global__ void __launch_bounds__(192) k_stage_tc_ring(TcArgs a) {
  using namespace tc;
  constexpr bool BF16 = MODE == kTcBF16;
  constexpr bool X3 = MODE == kTcX3;
  constexpr uint32_t TA = X3 ? 32768u : 16384u;
  constexpr int ESZ = BF16 ? 4 : 8;  // bytes per complex entry of A
  constexpr int KC = 128 / ESZ;      // complex columns per 128-byte chunk
  constexpr int CPC = 16 / ESZ;      // complex entries per 16-byte copy
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_full[S];
  __shared__ __align__(8) uint64_t s_bready[S];
  __shared__ __align__(8) uint64_t s_empty[S];
  __shared__ __align__(8) uint64_t s_done;
  extern __shared__ __align__(16) uint8_t smem_dyn[];
  const uint32_t base = (su32(smem_dyn) + 1023u) & ~1023u;
  uint8_t* gbase = smem_dyn + (base - su32(smem_dyn));
  const uint32_t TB = (uint32_t)a.nmax * 128;                  // one B tile (a multiple of 2048)
  const uint32_t SB = (uint32_t)tc_ring_stage_bytes(MODE, a.nmax);
  const uint32_t XOFF = TA + (X3 ? 2u : 1u) * TB;              // x staging inside a stage
  int* sIdx = reinterpret_cast<int*>(gbase + S * SB);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int2 t = a.tiles[blockIdx.x];
  const int blk = t.x, r0 = t.y * kTcRows;
  const int2 d = a.dims[blk];
  const int nrows = ADJ ? d.y : d.x, ncols = ADJ ? d.x : d.y;
  const int j0 = blockIdx.y * kTcMaxRhs;
  const int bcta = min(kTcMaxRhs, a.b - j0);
  const int bp = (bcta + 7) & ~7;
  const int N = 2 * bp;
  const int sld = a.nmax / 2;
  const uint32_t ncol_tmem = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  const int* rowidx = a.rowidx + (size_t)blk * (ADJ ? a.ldc : a.ldr);
  const int* colidx = a.colidx + (size_t)blk * (ADJ ? a.ldr : a.ldc);
  const uint8_t* Ab = (const uint8_t*)a.A + (size_t)blk * a.bstride * ESZ;
  const uint32_t id = idesc(BF16 ? 1u : 2u, kTcRows, N);
  const int nchunks = (ncols + KC - 1) / KC;

  if (warp == 0) tmem_alloc(&s_tmem, ncol_tmem);
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&s_full[q], 32);
      mbar_init(&s_bready[q], 128);
      mbar_init(&s_empty[q], 1);
    }
    mbar_init(&s_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < ncols; e += 192) sIdx[e] = colidx[e];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  bool ok = true;
  if (warp == 4) {
    // producer
    for (int k = 0; k < nchunks && ok; ++k) {
      const int st = k % S;
      if (k >= S) ok = mbar_wait(&s_empty[st], (uint32_t)((k / S - 1) & 1));
      if (!ok) break;
      const uint32_t sA = base + st * SB, sX = sA + XOFF;
      const int c0 = k * KC;
      for (int e = lane; e < kTcRows * 8; e += 32) {
        const int row = e >> 3, ch = e & 7;
        const int gr = r0 + row, gc = c0 + ch * CPC;
        const bool in = gr < nrows && gc < ncols;
        const void* src = in ? (const void*)(Ab + ((size_t)gr * a.lda + gc) * ESZ) : a.A;
        cp16(sA + swz(row, ch), src, in ? 16 : 0);
      }
      if (a.stage_x) {
        const int cpr = bcta >> 1;
        for (int e = lane; e < KC * cpr; e += 32) {
          const int c = e / cpr, q = e - c * cpr;
          const int idx = (c0 + c < ncols) ? sIdx[c0 + c] : -1;
          const void* src = idx >= 0 ? (const void*)(a.x + (long long)idx * a.xrs + j0 + 2 * q) : (const void*)a.x;
          cp16(sX + (uint32_t)((c * sld + 2 * q) * 8), src, idx >= 0 ? 16 : 0);
        }
      }
      cp_mbar_arrive(&s_full[st]);
    }
    cp_wait_all();
  } else if (warp == 5) {
    // MMA issuer
    if (lane == 0) {
      for (int k = 0; k < nchunks && ok; ++k) {
        const int st = k % S;
        ok = mbar_wait(&s_bready[st], (uint32_t)((k / S) & 1));
        if (!ok) break;
        fence_after();
        const uint32_t sA = base + st * SB, sB = sA + TA;
        if (X3) {  // the same order as k_stage_tc
#pragma unroll
          for (int q = 0; q < 4; ++q)
            mma<false>(tmem, sdesc(sA + 16384 + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            mma<false>(tmem, sdesc(sA + 32 * q), sdesc(sB + TB + 32 * q), id, 1u);
            mma<false>(tmem, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, 1u);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            mma<BF16>(tmem, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
        }
        mma_commit(&s_empty[st]);
      }
      if (nchunks > 0) {
        // every MMA issued so far is finished before `done` completes (also after a timeout)
        mma_commit(&s_done);
        ok = mbar_wait(&s_done, 0) && ok;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  } else {
    // warps 0-3: B expansion (and the A split), then the epilogue
    for (int k = 0; k < nchunks && ok; ++k) {
      const int st = k % S;
      ok = mbar_wait(&s_full[st], (uint32_t)((k / S) & 1));
      if (!ok) break;
      uint8_t* pA = gbase + st * SB;
      uint8_t* pB = pA + TA;
      const float2* pX = reinterpret_cast<const float2*>(pA + XOFF);
      const int c0 = k * KC;
      for (int e = tid; e < KC * bp; e += 128) {
        const int c = e / bp, j = e - c * bp;
        float2 v = make_float2(0.f, 0.f);
        if (j < bcta) {
          if (a.stage_x) {
            v = pX[c * sld + j];
          } else if (c0 + c < ncols) {
            const int idx = sIdx[c0 + c];
            if (idx >= 0) v = a.x[(long long)idx * a.xrs + (long long)(j0 + j) * a.xcs];
          }
        }
        float p0, p1, q0, q1;
        if (!ADJ) {
          p0 = v.x; p1 = -v.y; q0 = v.y; q1 = v.x;
        } else {
          p0 = v.x; p1 = v.y; q0 = v.y; q1 = -v.x;
        }
        const int n0 = 2 * j, n1 = 2 * j + 1;
        if (BF16) {
          const int ch = c >> 2, off = (c & 3) << 2;
          *reinterpret_cast<__nv_bfloat162*>(pB + swz(n0, ch) + off) = __floats2bfloat162_rn(p0, p1);
          *reinterpret_cast<__nv_bfloat162*>(pB + swz(n1, ch) + off) = __floats2bfloat162_rn(q0, q1);
        } else if (X3) {
          const int ch = c >> 1, off = (c & 1) << 3;
          const float hp0 = tf32_rna(p0), hp1 = tf32_rna(p1), hq0 = tf32_rna(q0), hq1 = tf32_rna(q1);
          *reinterpret_cast<float2*>(pB + swz(n0, ch) + off) = make_float2(hp0, hp1);
          *reinterpret_cast<float2*>(pB + swz(n1, ch) + off) = make_float2(hq0, hq1);
          *reinterpret_cast<float2*>(pB + TB + swz(n0, ch) + off) =
              make_float2(tf32_rna(p0 - hp0), tf32_rna(p1 - hp1));
          *reinterpret_cast<float2*>(pB + TB + swz(n1, ch) + off) =
              make_float2(tf32_rna(q0 - hq0), tf32_rna(q1 - hq1));
        } else {
          const int ch = c >> 1, off = (c & 1) << 3;
          *reinterpret_cast<float2*>(pB + swz(n0, ch) + off) = make_float2(p0, p1);
          *reinterpret_cast<float2*>(pB + swz(n1, ch) + off) = make_float2(q0, q1);
        }
      }
      if (X3) {
        for (int e = tid; e < kTcRows * 8; e += 128) {
          float4* h = reinterpret_cast<float4*>(pA + 16 * e);
          const float4 v = *h;
          const float4 hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
          *h = hi;
          *reinterpret_cast<float4*>(pA + 16384 + 16 * e) =
              make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z), tf32_rna(v.w - hi.w));
        }
      }
      fence_async_smem();
      mbar_arrive(&s_bready[st]);
    }
    if (nchunks > 0 && ok) ok = mbar_wait(&s_done, 0);
    fence_after();
    // epilogue: warp w holds accumulator rows 32w .. 32w+31 (TMEM lanes)
    const int row = r0 + warp * 32 + lane;
    const int oidx = (row < nrows) ? rowidx[row] : -1;
    for (int cb = 0; cb < N; cb += 16) {
      uint32_t r[16];
      if (nchunks > 0 && ok) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0u;
      }
      if (oidx >= 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = cb / 2 + q;
          if (j < bcta)
            a.y[(long long)oidx * a.yrs + (long long)(j0 + j) * a.ycs] =
                make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
        }
      }
    }
  }
  if (!ok) atomicExch(&g_tc_timeout, 1);
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncol_tmem);
}

// Self-test of the bounded wait: every CTA waits on an mbarrier that nothing arrives at, with a
// limit of limit_ns; the wait must give up, record the timeout and return.
__global__ void k_wait_selftest(uint64_t limit_ns, int* gave_up) {
  using namespace tc;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) {
    atomicAdd(gave_up, 1);
    atomicExch(&g_tc_timeout, 1);
  }
}

// block-wise transpose of the complex64 copy: out block (C x R) = in block (R x C)^T
__global__ void k_transpose_blocks(const float2* in, float2* out, int nblk, int R, int C) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)R * C;
  if (t >= per * nblk) return;
  const long long b = t / per, e = t - b * per;
  const int r = (int)(e / C), c = (int)(e - (long long)r * C);
  out[b * per + (long long)c * R + r] = in[t];
}

// bf16 copy with row stride ld (>= cols, padding zero): out[b][r][0..ld) from in[b][r][0..cols)
__global__ void k_to_bf16(const float2* in, __nv_bfloat162* out, int nblk, int rows, int cols, int ld) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)rows * ld;
  if (t >= per * nblk) return;
  const long long b = t / per, e = t - b * per;
  const int r = (int)(e / ld), c = (int)(e - (long long)r * ld);
  const float2 v = c < cols ? in[b * (long long)rows * cols + (long long)r * cols + c] : make_float2(0.f, 0.f);
  out[t] = __floats2bfloat162_rn(v.x, v.y);
}

}  // namespace fio

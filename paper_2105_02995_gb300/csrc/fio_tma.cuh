// fio_tma.cuh -- persistent, warp-specialised tcgen05 stage kernel whose factor tiles arrive by
// TMA (cp.async.bulk.tensor), for batched right-hand sides on sm_103a.
//
// The product of one stage block is the real GEMM of fio_tc.cuh (the block's complex rows read
// as interleaved reals are the K-major A operand; the gathered x rows are expanded into the B^T
// tile with the forward or adjoint sign pattern; the (re, im) pair of output (r, j) lands in
// accumulator columns 2j, 2j+1 of row r).  What differs is how the factor -- the only large
// operand, read once per apply -- is streamed:
//   * A tiles (128 rows x 128 bytes of K) come by TMA from a 2D tensor map over the stage's
//     factor array ([nblk * rows] x [2 * lda] reals, 128-byte swizzle, the canonical K-major
//     layout of the MMA) as up to four boxes of 32 rows, stopping at the block's last valid row
//     (the swizzle depends on the shared-memory address only, so four 32-row boxes land exactly
//     as one 128-row box would; rows past the block are never read from HBM and their
//     accumulator rows are never stored), into a ring of SA slots sized at launch to what shared
//     memory holds (up to 11 x 16 KB: under load an HBM round trip takes microseconds, and the
//     ring has to keep ~130 KB per SM in flight to stream at the copy rate), with an L2
//     evict-first policy so that the factor stream does not push the stage vectors out of L2;
//   * the CTA is persistent (one per SM) and walks a list of work units (block, first 128-row
//     tile, up to G tiles) sorted by size; all tiles of a unit share the chunk's B tile, so the x
//     gather and the B expansion are done once per chunk for up to G row tiles;
//   * warp roles: warp 0 issues the TMA loads; warp 1 issues the MMAs (one elected lane);
//     warps 2-5 gather the chunk's x rows (16-byte cp.async, up to seven chunks ahead, their gather
//     indices loaded one chunk earlier still; every thread expands the entries it copied itself,
//     so no barrier couples the 128 threads) and expand them into the B tile; warps 6-9 read the
//     accumulators out of tensor memory and scatter the rows; in split-TF32 mode warps 10-13
//     split the landed A tiles into head (in place) and tail (a ring of its own, so every A slot
//     is a TMA target);
//   * accumulators are double-buffered in tensor memory (2 x 256 columns: all of an SM's tensor
//     memory, so one CTA per SM), so the epilogue of a unit overlaps the MMAs of the next.
// Every wait is bounded by %globaltimer (kWaitNs); a role whose wait gives up stops, records the
// timeout in g_tc_timeout, and the CTA still waits (bounded) for its TMA loads, copies and MMAs
// before tensor memory is freed.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fio_tc.cuh"

namespace fio {

struct TmaArgs {
  const int* rowidx;  // output index lists (forward: out, adjoint: in), block stride lrow
  const int* colidx;  // gather index lists (forward: in, adjoint: out), block stride lcol
  int lrow, lcol;
  int rows_per_blk;   // rows of one block in the A tensor (forward R, adjoint C)
  const int2* dims;   // per block (valid rows, valid cols) of the forward block
  const int4* units;  // (block, first 128-row tile, tiles) per work unit
  int nunits;
  int nrhs_tiles;     // ceil(b / 64)
  const float2* x;    // row-major work vector: x[idx * xrs + j]
  long long xrs;
  float2* y;
  long long yrs, ycs;
  int b;
  int nmax;           // accumulator columns of a full right-hand-side tile (2 x RHS padded to 8)
  int ksplit;         // every block's chunks split into ksplit slices, one work unit each (>= 1)
  float2* part;       // null: rows go to y; else slice ks of row r of block blk goes to
                      // part[(ks * prow + blk * rows_per_blk + r) * b + j] (summed by k_partial_reduce)
  long long prow;     // rows of one slice of `part` (nblk * rows_per_blk)
  int sa;             // A ring slots (1 .. kMaxSA), set by the launcher from the shared memory
  int sx;             // x staging slots (3 .. kMaxSX): gathers run sx - 1 chunks ahead
  int sl;             // split mode: tail ring slots (2 .. kMaxSL)
};

namespace tma {

constexpr int kThreads = 448;  // 14 warps: producer, MMA, 4 expanders, 4 epilogue, 4 splitters
constexpr uint32_t kTmemCols = 512;  // two accumulator buffers of 256 columns
constexpr uint32_t kBufCols = kTmemCols / 2;
constexpr int kBoxRows = 32;         // rows per TMA box (four boxes fill one 128-row tile)
constexpr uint32_t kATile = 16384;   // one 128 x 128-byte A tile
constexpr int kMaxSX = 8;            // x staging slots at most (gathers run up to 7 chunks ahead)
constexpr int kMaxSA = 11;           // A ring slots at most
constexpr int kMaxSL = 6;            // split mode: slots of the tail tiles at most
constexpr int kMaxPf = 8;            // gather copies per thread and chunk at most (KC x b / 2 / 128)

template <int MODE> struct Cfg {
  static constexpr bool BF16 = MODE == kTcBF16, X3 = MODE == kTcX3;
  static constexpr int SB = X3 ? 2 : 3;                     // B ring stages
  static constexpr int KC = BF16 ? 32 : 16;                 // complex columns per 128-byte chunk
};

// dynamic shared memory besides the A ring, the tail ring and the x staging, for accumulator
// width nmax: alignment slack and the B ring; and one x staging slot
__host__ __device__ constexpr int smem_fixed(int mode, int nmax) {
  return 1024 + (mode == kTcX3 ? 2 * 2 : 3) * nmax * 128;
}
__host__ __device__ constexpr int xslot_bytes(int mode, int nmax) { return (mode == kTcBF16 ? 32 : 16) * (nmax / 2) * 8; }
__host__ __device__ constexpr int smem_bytes(int mode, int nmax, int sa, int sx, int sl) {
  return smem_fixed(mode, nmax) + (sa + (mode == kTcX3 ? sl : 0)) * 16384 + sx * xslot_bytes(mode, nmax);
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int cx, int cy, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cx), "r"(cy), "r"(tc::su32(bar)), "l"(policy)
      : "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// all but the newest n (0 .. kMaxSX - 2) commit groups of this thread have landed
__device__ __forceinline__ void cp_wait_newest(int n) {
  switch (n) {
    case 0: cp_wait_group<0>(); break;
    case 1: cp_wait_group<1>(); break;
    case 2: cp_wait_group<2>(); break;
    case 3: cp_wait_group<3>(); break;
    case 4: cp_wait_group<4>(); break;
    case 5: cp_wait_group<5>(); break;
    default: cp_wait_group<6>(); break;
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// work unit u of the CTA's sequence: unit list entry, chunk slice and right-hand-side tile
struct Unit {
  int blk, t0, nt, j0, bcta, N, nrows, ncols, ks, kb, nchunks;
};
template <bool ADJ, int KC>
__device__ __forceinline__ Unit unit_at(const TmaArgs& a, int u) {
  Unit w;
  const int per = a.nunits * a.ksplit;
  const int rt = u / per, rem = u - rt * per;
  w.ks = rem / a.nunits;
  const int ui = rem - w.ks * a.nunits;
  const int4 e = a.units[ui];
  w.blk = e.x;
  w.t0 = e.y;
  w.nt = e.z;
  w.j0 = rt * kTcMaxRhs;
  w.bcta = min(kTcMaxRhs, a.b - w.j0);
  w.N = 2 * ((w.bcta + 7) & ~7);
  const int2 d = a.dims[w.blk];
  w.nrows = ADJ ? d.y : d.x;
  w.ncols = ADJ ? d.x : d.y;
  const int nch = (w.ncols + KC - 1) / KC;          // chunks of the block
  const int cps = (nch + a.ksplit - 1) / a.ksplit;  // chunks per slice
  w.kb = min(nch, w.ks * cps);
  w.nchunks = min(nch, w.kb + cps) - w.kb;          // may be 0: the slice then stores zeros
  return w;
}

}  // namespace tma

template <bool ADJ, int MODE>
__global__ void __launch_bounds__(tma::kThreads, 1) k_stage_tma(const TmaArgs a, const __grid_constant__ CUtensorMap amap) {
  using namespace tc;
  using namespace tma;
  using C = Cfg<MODE>;
  constexpr int SB = C::SB, KC = C::KC;
  constexpr bool BF16 = C::BF16, X3 = C::X3;
  const int SA = a.sa;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t a_full[kMaxSA], a_ready[kMaxSA], a_empty[kMaxSA];
  __shared__ __align__(8) uint64_t l_free[kMaxSL];  // split mode: a tail slot's MMAs are done
  __shared__ __align__(8) uint64_t b_full[SB], b_empty[SB];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], s_done;
  extern __shared__ __align__(16) uint8_t smem_dyn[];
  const uint32_t base = (su32(smem_dyn) + 1023u) & ~1023u;
  uint8_t* gbase = smem_dyn + (base - su32(smem_dyn));
  const uint32_t TB = (uint32_t)a.nmax * 128;            // one B tile (N rows x 128 bytes)
  const uint32_t BSTAGE = (X3 ? 2u : 1u) * TB;           // split mode: head tile + tail tile
  // layout: A ring (SA x 16 KB), tail ring (split mode), B ring, x staging
  const uint32_t OFF_L = (uint32_t)SA * kATile;
  const int SL = a.sl;
  const uint32_t OFF_B = OFF_L + (X3 ? (uint32_t)SL * kATile : 0u), OFF_X = OFF_B + SB * BSTAGE;
  const int sld = a.nmax / 2;                             // staging row length (complex)
  const uint32_t XSLOT = (uint32_t)(KC * sld * 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = a.nunits * a.ksplit * a.nrhs_tiles;

  if (warp == 0) tmem_alloc(&s_tmem, kTmemCols);
  if (tid == 0) {
    for (int q = 0; q < SA; ++q) {
      mbar_init(&a_full[q], 1);
      mbar_init(&a_ready[q], 128);
      mbar_init(&a_empty[q], 1);
    }
    for (int q = 0; q < SB; ++q) {
      mbar_init(&b_full[q], 128);
      mbar_init(&b_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 128);
    }
    for (int q = 0; q < kMaxSL; ++q) mbar_init(&l_free[q], 1);
    mbar_init(&s_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  bool ok = true;

  if (warp == 0) {
    // ---- TMA producer ------------------------------------------------------------------------
    if (lane == 0) {
      const uint64_t pol = evict_first_policy();
      uint32_t ia = 0;
      for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
        const Unit w = unit_at<ADJ, KC>(a, u);
        const int row0 = w.blk * a.rows_per_blk + w.t0 * kTcRows;
        for (int k = 0; k < w.nchunks && ok; ++k) {
          for (int t = 0; t < w.nt; ++t, ++ia) {
            const int s = (int)(ia % SA);
            if (ia >= (uint32_t)SA && !mbar_wait(&a_empty[s], ((ia / SA) - 1) & 1)) {
              ok = false;
              break;
            }
            // boxes of 32 rows up to the block's last valid row (at least one: the tile exists)
            const int left = w.nrows - (w.t0 + t) * kTcRows;
            const int nbox = min(kTcRows / kBoxRows, (left + kBoxRows - 1) / kBoxRows);
            expect_tx(&a_full[s], (uint32_t)nbox * (kATile / (kTcRows / kBoxRows)));
            for (int q = 0; q < nbox; ++q)
              tma_load_2d(base + s * kATile + q * (kATile / (kTcRows / kBoxRows)), &amap,
                          (w.kb + k) * 64 / (BF16 ? 1 : 2), row0 + t * kTcRows + q * kBoxRows, &a_full[s], pol);
          }
        }
      }
      // every load issued has landed before the CTA may leave (after a timeout as well)
      for (uint32_t i = ia > (uint32_t)SA ? ia - SA : 0; i < ia; ++i)
        if (!mbar_wait(&a_full[i % SA], (i / SA) & 1)) ok = false;
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer --------------------------------------------------------------------------
    if (lane == 0) {
      uint32_t ia = 0, ib = 0, v = 0;
      for (int u = blockIdx.x; u < total && ok; u += gridDim.x, ++v) {
        const Unit w = unit_at<ADJ, KC>(a, u);
        const uint32_t buf = v & 1;
        const uint32_t id = idesc(BF16 ? 1u : 2u, kTcRows, w.N);
        if (v >= 2 && !mbar_wait(&acc_empty[buf], ((v / 2) - 1) & 1)) {
          ok = false;
          break;
        }
        fence_after();
        for (int k = 0; k < w.nchunks && ok; ++k, ++ib) {
          const int sb = (int)(ib % SB);
          if (!mbar_wait(&b_full[sb], (ib / SB) & 1)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sB = base + OFF_B + sb * BSTAGE;
          for (int t = 0; t < w.nt; ++t, ++ia) {
            const int s = (int)(ia % SA);
            if (!mbar_wait(X3 ? &a_ready[s] : &a_full[s], (ia / SA) & 1)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t sA = base + s * kATile;
            const uint32_t sL = base + OFF_L + (ia % SL) * kATile;  // split mode: tail tile
            const uint32_t d = tmem + buf * kBufCols + (uint32_t)(t * w.N);
            if (X3) {
              // the tail tile's products first, committed on their own so that the tail slot is
              // free for the next split as soon as they are done; then the head products
#pragma unroll
              for (int q = 0; q < 4; ++q)
                mma<false>(d, sdesc(sL + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
              mma_commit(&l_free[ia % SL]);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                mma<false>(d, sdesc(sA + 32 * q), sdesc(sB + TB + 32 * q), id, 1u);
                mma<false>(d, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, 1u);
              }
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                mma<BF16>(d, sdesc(sA + 32 * q), sdesc(sB + 32 * q), id, (k > 0 || q > 0) ? 1u : 0u);
            }
            mma_commit(&a_empty[s]);
          }
          if (ok) mma_commit(&b_empty[sb]);
        }
        if (ok) mma_commit(&acc_full[buf]);
      }
      // every MMA issued is finished before the tiles and tensor memory are released
      mma_commit(&s_done);
      if (!mbar_wait(&s_done, 0)) ok = false;
    }
    __syncwarp();
  } else if (warp < 6) {
    // ---- x gather, B expansion (and the A split) --------------------------------------------
    // Each of the 128 threads owns pairs (gathered row c, right-hand sides 2q and 2q+1): pair
    // p = c * HP + q with HP = nmax / 4 (the pairs of a full right-hand-side tile, the same for
    // every unit of the launch, so that a thread owns the same staging entries whatever the
    // unit's width) belongs to thread p mod 128.  It issues that pair's 16-byte copy into the
    // staging slot and later expands those two entries into the B tile, so it only ever reads its
    // own copies -- its own cp.async.wait_group is the only synchronisation the staging needs, and
    // the threads run without a group barrier (a thread whose bounded wait gives up stops
    // arriving; the MMA warp's wait then gives up too).
    // The gather of a chunk takes two steps: pf_load reads the chunk's gather indices into
    // registers, pf_issue -- one expansion later, so that the index loads are long done -- issues
    // the copies; the copies run two chunks ahead of the expansion.
    const int et = tid - 64;
    const int HP = a.nmax >> 2;   // pairs per gathered row of a full right-hand-side tile
    int fu = blockIdx.x, fk = 0;  // fetch cursor: unit and chunk of the next pf_load
    Unit fw{};
    if (fu < total) fw = unit_at<ADJ, KC>(a, fu);
    int pf_idx[kMaxPf];
    int pf_cpr = 0, pf_j0 = 0;
    bool pf_live = false;
    auto pf_load = [&]() {
      while (fu < total && fk >= fw.nchunks) {  // skip units without chunks
        fu += gridDim.x;
        fk = 0;
        if (fu < total) fw = unit_at<ADJ, KC>(a, fu);
      }
      pf_live = fu < total;
      if (!pf_live) return;
      const int* cidx = a.colidx + (size_t)fw.blk * a.lcol;
      pf_cpr = fw.bcta >> 1;   // pairs that hold data
      pf_j0 = fw.j0;
#pragma unroll
      for (int m = 0; m < kMaxPf; ++m) {
        const int p = et + 128 * m;
        int idx = -1;
        if (p < KC * HP) {
          const int c = p / HP, q = p - c * HP;
          const int col = (fw.kb + fk) * KC + c;
          if (q < pf_cpr && col < fw.ncols) idx = cidx[col];
        }
        pf_idx[m] = idx;
      }
      ++fk;
    };
    auto pf_issue = [&](uint32_t slot) {
      if (pf_live) {
        const uint32_t dst = base + OFF_X + slot * XSLOT;
#pragma unroll
        for (int m = 0; m < kMaxPf; ++m) {
          const int p = et + 128 * m;
          if (p < KC * HP) {
            const int c = p / HP, q = p - c * HP;
            if (q < pf_cpr) {
              const int idx = pf_idx[m];
              const void* src = idx >= 0 ? (const void*)(a.x + (long long)idx * a.xrs + pf_j0 + 2 * q) : (const void*)a.x;
              cp16(dst + (uint32_t)((c * sld + 2 * q) * 8), src, idx >= 0 ? 16 : 0);
            }
          }
        }
      }
      cp_commit();
    };
    const int SX = a.sx, D = SX - 1;  // gathers run D chunks ahead of the expansion
    for (int q = 0; q < D; ++q) {
      pf_load();
      pf_issue((uint32_t)q);
    }
    pf_load();
    uint32_t ia = 0, ib = 0;
    int u = blockIdx.x, k = 0;  // cursor of the chunk being expanded
    Unit w{};
    if (u < total) w = unit_at<ADJ, KC>(a, u);
    while (ok) {
      while (u < total && k >= w.nchunks) {
        u += gridDim.x;
        k = 0;
        if (u < total) w = unit_at<ADJ, KC>(a, u);
      }
      if (u >= total) break;
      cp_wait_newest(D - 1);     // this thread's copies of chunk ib have landed
      pf_issue((ib + D) % SX);   // chunk ib + D, its indices loaded one iteration ago
      pf_load();                 // indices of chunk ib + D + 1, in flight during the expansion
      const int sb = (int)(ib % SB);
      if (ib >= (uint32_t)SB) ok = mbar_wait(&b_empty[sb], ((ib / SB) - 1) & 1);
      if (!ok) break;
      uint8_t* pB = gbase + OFF_B + sb * BSTAGE;
      const float2* pX = reinterpret_cast<const float2*>(gbase + OFF_X + (ib % SX) * XSLOT);
      const int half = w.N >> 2;  // pairs of this unit's right-hand-side tile (<= HP)
      for (int p = et; p < KC * HP; p += 128) {
        const int c = p / HP, q = p - c * HP;
        if (q >= half) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * q + h;
          const float2 v = j < w.bcta ? pX[c * sld + j] : make_float2(0.f, 0.f);
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
            *reinterpret_cast<float2*>(pB + TB + swz(n0, ch) + off) = make_float2(tf32_rna(p0 - hp0), tf32_rna(p1 - hp1));
            *reinterpret_cast<float2*>(pB + TB + swz(n1, ch) + off) = make_float2(tf32_rna(q0 - hq0), tf32_rna(q1 - hq1));
          } else {
            const int ch = c >> 1, off = (c & 1) << 3;
            *reinterpret_cast<float2*>(pB + swz(n0, ch) + off) = make_float2(p0, p1);
            *reinterpret_cast<float2*>(pB + swz(n1, ch) + off) = make_float2(q0, q1);
          }
        }
      }
      fence_async_smem();
      mbar_arrive(&b_full[sb]);
      ++k;
      ++ib;
    }
    cp_wait_all();
  } else if (warp < 10) {
    // ---- epilogue: tensor memory -> scattered output rows -------------------------------------
    const int quad = warp & 3;  // TMEM lane quadrant this warp may read
    const bool to_part = a.part != nullptr;
    const bool vec_store = to_part || (a.ycs == 1 && (a.yrs & 1) == 0 && ((uintptr_t)a.y & 15) == 0);
    uint32_t v = 0;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x, ++v) {
      const Unit w = unit_at<ADJ, KC>(a, u);
      const uint32_t buf = v & 1;
      // the warp's lanes agree before the warp-collective tensor-memory loads
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (v / 2) & 1) ? 1 : 0)) {
        ok = false;
        break;
      }
      fence_after();
      const int* ridx = a.rowidx + (size_t)w.blk * a.lrow;
      for (int t = 0; t < w.nt; ++t) {
        const int row = (w.t0 + t) * kTcRows + quad * 32 + lane;
        const int oidx = row < w.nrows ? ridx[row] : -1;
        // destination row: the output row, or this slice's partial row of the block row
        float2* yr = to_part ? a.part + ((long long)w.ks * a.prow + (long long)w.blk * a.rows_per_blk + row) * a.b
                             : a.y + (long long)(oidx < 0 ? 0 : oidx) * a.yrs;
        for (int cb = 0; cb < w.N; cb += 16) {
          uint32_t r[16];
          if (w.nchunks > 0) {
            tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + buf * kBufCols + (uint32_t)(t * w.N + cb), r);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) r[q] = 0u;
          }
          if (oidx >= 0) {
            const int jb = cb / 2;
            if (vec_store && jb + 8 <= w.bcta) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                *reinterpret_cast<float4*>(yr + w.j0 + jb + 2 * q) =
                    make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                                __uint_as_float(r[4 * q + 3]));
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q)
                if (jb + q < w.bcta)
                  yr[(long long)(w.j0 + jb + q) * (to_part ? 1 : a.ycs)] =
                      make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
  } else if (X3) {
    // ---- split-TF32: every landed A tile split into head (in place) and tail (tail ring) -----
    const int et = tid - 320;
    uint32_t ia = 0;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const Unit w = unit_at<ADJ, KC>(a, u);
      for (int k = 0; k < w.nchunks && ok; ++k) {
        for (int t = 0; t < w.nt; ++t, ++ia) {
          const int s = (int)(ia % SA);
          ok = mbar_wait(&a_full[s], (ia / SA) & 1);
          // the tail slot was last used by tile ia - SL, whose tail products released it
          if (ok && ia >= (uint32_t)SL) ok = mbar_wait(&l_free[ia % SL], ((ia / SL) - 1) & 1);
          if (!ok) break;
          uint8_t* pA = gbase + s * kATile;
          uint8_t* pL = gbase + OFF_L + (ia % SL) * kATile;
          for (int e = et; e < (int)(kATile / 16); e += 128) {
            float4* hp = reinterpret_cast<float4*>(pA + 16 * e);
            const float4 v = *hp;
            const float4 hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
            *hp = hi;
            *reinterpret_cast<float4*>(pL + 16 * e) =
                make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z), tf32_rna(v.w - hi.w));
          }
          fence_async_smem();
          mbar_arrive(&a_ready[s]);
        }
      }
    }
  }

  if (!ok) atomicExch(&g_tc_timeout, 1);
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// The slices of a split in-place stage summed in slice order, written into the work vector W at
// the block rows' own indices (the in-place stage's copy-back): W[idx[r]][j] = sum_ks part[ks][r][j]
// for every packed row r of the stage with idx[r] >= 0 (the blocks' index sets are disjoint).
__global__ void k_partial_reduce(const float2* part, int ksplit, long long prow, int b, const int* idx, float2* W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prow * b) return;
  const long long r = t / b;
  const int j = (int)(t - r * b);
  const int row = idx[r];
  if (row < 0) return;
  float2 acc = part[t];
  for (int q = 1; q < ksplit; ++q) {
    const float2 v = part[(long long)q * prow * b + t];
    acc.x += v.x;
    acc.y += v.y;
  }
  W[(long long)row * b + j] = acc;
}

}  // namespace fio

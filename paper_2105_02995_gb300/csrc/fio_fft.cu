// fio_fft.cu -- the DFT F of the paper's problem statement (section 1) and its inverse, on the
// device: u = K F f, so the full solve is f = F^{-1} (K^{-1} u), and F is the step after the
// approximate inverse.
//
//   F      f-hat(xi) = n^{-d} sum_x exp(-2 pi i x.xi) f(x)       (section 1, the DFT of f)
//   F^{-1} f(x)      =         sum_xi exp(+2 pi i x.xi) f-hat(xi)
// on the grids x = k/n, xi = j - n/2 per dimension (2D index i1 + n*i2).  With xi = j - n/2,
// exp(-+2 pi i x.xi) = (-1)^(k_1+..+k_d) exp(-+2 pi i k.j/n): F is the standard DFT of the
// sign-modulated input scaled by n^{-d}, F^{-1} the sign-modulated standard inverse DFT.
//
// Kernel: k_fft_pass, a batch of power-of-two transforms of length L <= 2048 in shared memory,
// 2048 / L transforms per CTA (one right-hand side per grid row).  Element e of transform t is
// read at t*xt + e*xe and written at t*yt + e*ye of the right-hand side's vector, so one kernel
// serves the contiguous and the strided axes; the copies walk whichever index is contiguous in
// memory.  In shared memory: elements loaded to bit-reversed positions, then log2 L in-place
// radix-2 butterfly stages (twiddles from a per-CTA table of exp(s 2 pi i t/L), t < L/2).
// Optional per-element factors: the (-1)^k sign modulation on the input (F) or on the output
// (F^{-1}), the four-step twiddle exp(s 2 pi i t e / N) on the output, and a scale.
// Plans: 2D n x n = transforms along i1, then along i2; 1D N <= 2048 = one pass; 1D N > 2048 =
// four-step (N = N1 N2, N1 <= N2): length-N2 transforms over j2 with the twiddle, then length-N1
// transforms over j1 written to k2 + N2 k1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fio.h"
#include "fio_internal.h"

namespace {

constexpr int kFftElems = 2048;  // complex elements per CTA
constexpr int kFftThreads = 256;

struct FftPass {
  const void* x;
  void* y;
  long long ldx, ldy;  // per right-hand side
  int L, logL;         // transform length and log2
  int T;               // transforms per right-hand side
  long long xt, xe;    // input offset of element e of transform t: t*xt + e*xe
  long long yt, ye;    // output offset
  int sign;            // +1: exp(+2 pi i ...) (inverse DFT), -1: forward
  int twN;             // > 0: multiply output (t, e) by exp(sign 2 pi i (t e mod twN) / twN)
  int mod_in, mod_out; // (-1)^(grid coordinate sum) of the input / output linear index
  int n, logn, d;      // grid (for the modulation)
  double scale;        // output scale
};

template <typename R> struct Cplx;
template <> struct Cplx<float> {
  using T = float2;
  static __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ void sincospi_(float a, float* s, float* c) { sincospif(a, s, c); }
};
template <> struct Cplx<double> {
  using T = double2;
  static __device__ __forceinline__ T make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ void sincospi_(double a, double* s, double* c) { sincospi(a, s, c); }
};

__device__ __forceinline__ bool odd_coord_sum(long long k, const FftPass& p) {
  if (p.d == 1) return (k & 1) != 0;
  return (((k & (p.n - 1)) + (k >> p.logn)) & 1) != 0;
}

template <typename R>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(FftPass p) {
  using C = Cplx<R>;
  using V = typename C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s = reinterpret_cast<V*>(smem_raw);         // kFftElems
  V* tw = s + kFftElems;                        // L/2 twiddles
  const int L = p.L, TT = kFftElems / L;
  const int t0 = blockIdx.x * TT;
  const int j = blockIdx.y;
  const V* x = reinterpret_cast<const V*>(p.x) + (long long)j * p.ldx;
  V* y = reinterpret_cast<V*>(p.y) + (long long)j * p.ldy;
  const int tid = threadIdx.x;

  for (int q = tid; q < L / 2; q += kFftThreads) {
    R sn, cs;
    C::sincospi_((R)(2 * q) / (R)L, &sn, &cs);  // exact argument: 2q/L with L a power of two
    tw[q] = C::make(cs, (R)p.sign * sn);
  }
  // load: element (t, e) -> s[tl*L + bitrev(e)]; the contiguous index varies fastest
  const bool e_fast = p.xe == 1 || p.xt != 1;
  for (int i = tid; i < TT * L; i += kFftThreads) {
    int tl, e;
    if (e_fast) {
      tl = i / L;
      e = i - tl * L;
    } else {
      e = i / TT;
      tl = i - e * TT;
    }
    const int t = t0 + tl;
    V v = C::make(0, 0);
    if (t < p.T) {
      const long long k = (long long)t * p.xt + (long long)e * p.xe;
      v = x[k];
      if (p.mod_in && odd_coord_sum(k, p)) v = C::make(-v.x, -v.y);
    }
    s[tl * L + (int)(__brev((unsigned)e) >> (32 - p.logL))] = v;
  }
  __syncthreads();
  // radix-2 butterflies, in place, spans 1, 2, 4, ..., L/2
  for (int lh = 0; lh < p.logL; ++lh) {
    const int half = 1 << lh;
    for (int i = tid; i < TT * (L / 2); i += kFftThreads) {
      const int tl = i / (L / 2), r = i - tl * (L / 2);
      const int g = r >> lh, k = r & (half - 1);
      const int a0 = tl * L + (g << (lh + 1)) + k, a1 = a0 + half;
      const V w = tw[k << (p.logL - 1 - lh)];
      const V u = s[a0], v = s[a1];
      const V wv = C::make(w.x * v.x - w.y * v.y, w.x * v.y + w.y * v.x);
      s[a0] = C::make(u.x + wv.x, u.y + wv.y);
      s[a1] = C::make(u.x - wv.x, u.y - wv.y);
    }
    __syncthreads();
  }
  // store: frequency e of transform t
  const bool oe_fast = p.ye == 1 || p.yt != 1;
  for (int i = tid; i < TT * L; i += kFftThreads) {
    int tl, e;
    if (oe_fast) {
      tl = i / L;
      e = i - tl * L;
    } else {
      e = i / TT;
      tl = i - e * TT;
    }
    const int t = t0 + tl;
    if (t >= p.T) continue;
    V v = s[tl * L + e];
    if (p.twN > 0) {
      const long long r = ((long long)t * e) % p.twN;
      R sn, cs;
      C::sincospi_((R)(2 * r) / (R)p.twN, &sn, &cs);
      sn *= (R)p.sign;
      v = C::make(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
    }
    const long long k = (long long)t * p.yt + (long long)e * p.ye;
    R sc = (R)p.scale;
    if (p.mod_out && odd_coord_sum(k, p)) sc = -sc;
    y[k] = C::make(sc * v.x, sc * v.y);
  }
}

int ilog2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

template <typename R>
int run_pass(const FftPass& p, int b, cudaStream_t s) {
  const int TT = kFftElems / p.L;
  dim3 grid((unsigned)((p.T + TT - 1) / TT), (unsigned)b);
  const size_t smem = (size_t)(kFftElems + p.L / 2) * sizeof(typename Cplx<R>::T);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_fft_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return FIO_ECUDA;
  }
  k_fft_pass<R><<<grid, kFftThreads, smem, s>>>(p);
  return FIO_OK;
}

// y = F x (inverse = false) or F^{-1} x (inverse = true); tmp: N x b scratch (ld N)
template <typename R>
int apply_dft(fio_op op, bool inverse, const void* x, void* y, long long ld, int b, void* tmp, cudaStream_t s) {
  const int n = (int)op->n, d = op->d;
  const long long N = op->N;
  FftPass p{};
  p.sign = inverse ? 1 : -1;
  p.n = n;
  p.logn = ilog2(n);
  p.d = d;
  const double scale_last = inverse ? 1.0 : 1.0 / (double)N;
  int rc;
  if (d == 2 || N > kFftElems) {
    // two passes: (2D) along i1 then along i2; (1D four-step) over j2 with twiddle, then over j1
    const int L1 = d == 2 ? n : (int)(1LL << (ilog2(N) / 2)), L2 = (int)(N / L1);
    FftPass a = p, c = p;
    a.x = x;
    a.y = tmp;
    a.ldx = ld;
    a.ldy = N;
    a.mod_in = inverse ? 0 : 1;
    a.scale = 1.0;
    c.x = tmp;
    c.y = y;
    c.ldx = N;
    c.ldy = ld;
    c.mod_out = inverse ? 1 : 0;
    c.scale = scale_last;
    if (d == 2) {
      a.L = n, a.T = n, a.xt = n, a.xe = 1, a.yt = n, a.ye = 1;   // along i1 for each i2
      c.L = n, c.T = n, c.xt = 1, c.xe = n, c.yt = 1, c.ye = n;   // along i2 for each i1
    } else {
      a.L = L2, a.T = L1, a.xt = 1, a.xe = L1, a.yt = 1, a.ye = L1, a.twN = (int)N;  // j1 + L1 j2 -> j1 + L1 k2
      c.L = L1, c.T = L2, c.xt = L1, c.xe = 1, c.yt = 1, c.ye = L2;                  // -> k2 + L2 k1
    }
    a.logL = ilog2(a.L);
    c.logL = ilog2(c.L);
    if ((rc = run_pass<R>(a, b, s))) return rc;
    if ((rc = run_pass<R>(c, b, s))) return rc;
  } else {
    p.x = x;
    p.y = y;
    p.ldx = ld;
    p.ldy = ld;
    p.L = (int)N;
    p.logL = ilog2(N);
    p.T = 1;
    p.xt = p.yt = 0;
    p.xe = p.ye = 1;
    p.mod_in = inverse ? 0 : 1;
    p.mod_out = inverse ? 1 : 0;
    p.scale = scale_last;
    if ((rc = run_pass<R>(p, b, s))) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? FIO_OK : FIO_ECUDA;
}

int dft_entry(fio_op op, bool inverse, const void* x, void* y, int64_t ld, int b, int dtype, int precision,
              void* stream) {
  if (!op || b < 0 || b > 65535 || ld < (op ? op->N : 0)) return FIO_EINVAL;  // b: grid rows
  if (!((dtype == FIO_C128 && precision == FIO_P64) || (dtype == FIO_C64 && precision == FIO_P32)))
    return FIO_EINVAL;
  if (b > 0 && (!x || !y || x == y)) return FIO_EINVAL;
  const long long n = op->n;
  if (n < 2 || (n & (n - 1)) != 0 || op->N > (long long)kFftElems * kFftElems) return FIO_ENOTSUP;
  const size_t es = dtype == FIO_C128 ? 16 : 8;
  const size_t span = ((size_t)ld * (b > 0 ? b - 1 : 0) + op->N) * es;
  const uint8_t *xb = (const uint8_t*)x, *yb = (const uint8_t*)y;
  if (b > 0 && xb < yb + span && yb < xb + span) return FIO_EINVAL;  // overlap
  if (b == 0) return FIO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaGetLastError() != cudaSuccess) return FIO_ECUDA;
  void* bufs[5];
  int rc = fio_scratch(op, b, es, s, bufs);
  if (rc) return rc;
  return dtype == FIO_C128 ? apply_dft<double>(op, inverse, x, y, ld, b, bufs[4], s)
                           : apply_dft<float>(op, inverse, x, y, ld, b, bufs[4], s);
}

}  // namespace

extern "C" int fio_apply_F(fio_op op, const void* f, void* fhat, int64_t ld, int b, int dtype, int precision,
                           void* stream) {
  return dft_entry(op, false, f, fhat, ld, b, dtype, precision, stream);
}

extern "C" int fio_apply_Finv(fio_op op, const void* fhat, void* f, int64_t ld, int b, int dtype, int precision,
                              void* stream) {
  return dft_entry(op, true, fhat, f, ld, b, dtype, precision, stream);
}

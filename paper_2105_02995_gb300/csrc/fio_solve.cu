// fio_solve.cu -- iterative solvers of K-dot f = u on the device (paper section 5 and the
// experiments of section 6), with the approximate inverse as preconditioner.
//
//   PCG    CG on the Hermitian system K-dot* K-dot f = K-dot* u preconditioned with G-dot
//          (the paper's pcg(K-dot* K-dot, K-dot* u, G-dot)).  The true residual s = u - K-dot f is
//          carried along (s -= alpha K-dot p) so the stopping test ||s|| <= tol ||u|| costs no
//          extra apply.
//   GMRES  restarted GMRES on K-dot f = u right-preconditioned with P = G-dot K-dot*; classical
//          Gram-Schmidt applied twice, Givens rotations per right-hand side on the host.
//   IR     iterative refinement: r = u - K-dot f on FP64 vectors (FP64 or double-float stage
//          arithmetic), d = G-dot K-dot* r in the inner precision (FP64, FP32 or tensor-core
//          factors), f += d in FP64.
// Every right-hand side has its own scalars; all of them advance together, a converged one is
// frozen.  Reductions are FP64 and in a fixed order (one CTA per column, fixed tree), so the
// results do not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "fio.h"
#include "fio_internal.h"

namespace {

constexpr int kRedThreads = 512;

// out[j] = sum_i conj(a[i, j]) b[i, j]   (one CTA per column j, fixed reduction tree)
__global__ void k_coldot(const double2* a, const double2* b, long long N, long long lda,
                         long long ldb, double2* out) {
  __shared__ double sr[kRedThreads], si[kRedThreads];
  const int j = blockIdx.x;
  const double2* x = a + (long long)j * lda;
  const double2* y = b + (long long)j * ldb;
  double re = 0.0, im = 0.0;
  for (long long i = threadIdx.x; i < N; i += kRedThreads) {
    const double2 u = x[i], v = y[i];
    re += u.x * v.x + u.y * v.y;
    im += u.x * v.y - u.y * v.x;
  }
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = make_double2(sr[0], si[0]);
}

// H[i + (k+1) j] = <V_i[:, j], w[:, j]> for i <= k   (grid (k+1, b))
__global__ void k_basisdot(const double2* V, long long vstride, const double2* w, long long N,
                           int b, int kp1, double2* H) {
  __shared__ double sr[kRedThreads], si[kRedThreads];
  const int i = blockIdx.x, j = blockIdx.y;
  const double2* x = V + (long long)i * vstride + (long long)j * N;
  const double2* y = w + (long long)j * N;
  double re = 0.0, im = 0.0;
  for (long long t = threadIdx.x; t < N; t += kRedThreads) {
    const double2 u = x[t], v = y[t];
    re += u.x * v.x + u.y * v.y;
    im += u.x * v.y - u.y * v.x;
  }
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) H[i + (long long)kp1 * j] = make_double2(sr[0], si[0]);
}

// w[:, j] -= sum_{i<=k} H[i + kp1 j] V_i[:, j]
__global__ void k_basis_sub(const double2* V, long long vstride, double2* w, long long N, int b,
                            int kp1, const double2* H) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * b) return;
  const int j = (int)(t / N);
  const long long r = t - (long long)j * N;
  double2 acc = w[t];
  for (int i = 0; i < kp1; ++i) {
    const double2 h = H[i + (long long)kp1 * j];
    const double2 v = V[(long long)i * vstride + (long long)j * N + r];
    acc.x -= h.x * v.x - h.y * v.y;
    acc.y -= h.x * v.y + h.y * v.x;
  }
  w[t] = acc;
}

// y[:, j] = alpha[j] x[:, j] + beta[j] y[:, j]   (x, y with leading dimensions)
__global__ void k_axpby(const double2* alpha, const double2* x, long long ldx, const double2* beta,
                        double2* y, long long ldy, long long N, int b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * b) return;
  const int j = (int)(t / N);
  const long long i = t - (long long)j * N;
  const double2 a = alpha[j], bb = beta[j];
  const double2 xv = x[i + j * ldx], yv = y[i + j * ldy];
  double2 r;
  r.x = a.x * xv.x - a.y * xv.y + bb.x * yv.x - bb.y * yv.y;
  r.y = a.x * xv.y + a.y * xv.x + bb.x * yv.y + bb.y * yv.x;
  y[i + j * ldy] = r;
}

__global__ void k_to32(const double2* x, float2* y, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = make_float2((float)x[t].x, (float)x[t].y);
}
__global__ void k_add32(const float2* d, double2* f, long long ldf, long long N, int b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * b) return;
  const int j = (int)(t / N);
  const long long i = t - (long long)j * N;
  f[i + j * ldf].x += (double)d[t].x;
  f[i + j * ldf].y += (double)d[t].y;
}

inline unsigned nblocks(long long n) { return (unsigned)((n + 255) / 256); }

struct Work {
  double2* v[6];       // N x b each, ld = N
  double2* basis;      // (restart + 1) x N x b
  double2* Hd;         // (restart + 1) x b scalars
  double2* sc;         // 4 x b scalars
  float2* v32[2];      // N x b
};

int get_work(fio_op op, int b, int restart, Work* w) {
  const long long N = op->N;
  const size_t vec = (size_t)N * b * sizeof(double2);
  const size_t need = 6 * vec + (size_t)(restart + 1) * vec + (size_t)(restart + 1) * b * sizeof(double2) +
                      4 * (size_t)b * sizeof(double2) + 2 * (size_t)N * b * sizeof(float2) + 1024;
  if (need > op->solver_bytes) {
    if (op->solver) cudaFree(op->solver);
    op->solver = nullptr;
    op->solver_bytes = 0;
    if (cudaMalloc(&op->solver, need) != cudaSuccess) {
      cudaGetLastError();
      return FIO_ENOMEM;
    }
    op->solver_bytes = need;
  }
  uint8_t* p = (uint8_t*)op->solver;
  for (int k = 0; k < 6; ++k) {
    w->v[k] = (double2*)p;
    p += vec;
  }
  w->basis = (double2*)p;
  p += (size_t)(restart + 1) * vec;
  w->Hd = (double2*)p;
  p += (size_t)(restart + 1) * b * sizeof(double2);
  w->sc = (double2*)p;
  p += 4 * (size_t)b * sizeof(double2);
  p = (uint8_t*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  w->v32[0] = (float2*)p;
  p += (size_t)N * b * sizeof(float2);
  w->v32[1] = (float2*)p;
  return FIO_OK;
}

struct Ctx {
  fio_op op;
  fio_op rop;           // operator of the true residuals (op itself, or a tighter butterfly)
  long long N;
  int b;
  cudaStream_t s;
  double2* dsc;         // device scalar scratch (4 x b)
  int outer = FIO_P64;  // precision of the true residuals (FIO_P64 or FIO_PDF)
  bool f_zero = false;  // f is known to be zero (the next residual is u itself)
};

int dots(Ctx& c, const double2* a, long long lda, const double2* bb, long long ldb, double2* out_dev,
         std::vector<double2>* host) {
  k_coldot<<<c.b, kRedThreads, 0, c.s>>>(a, bb, c.N, lda, ldb, out_dev);
  if (host) {
    host->resize(c.b);
    if (cudaMemcpyAsync(host->data(), out_dev, c.b * sizeof(double2), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
      return FIO_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? FIO_OK : FIO_ECUDA;
}

int axpby(Ctx& c, const std::vector<double2>& al, const double2* x, long long ldx,
          const std::vector<double2>& be, double2* y, long long ldy) {
  double2* d = c.dsc;
  cudaMemcpyAsync(d, al.data(), c.b * sizeof(double2), cudaMemcpyHostToDevice, c.s);
  cudaMemcpyAsync(d + c.b, be.data(), c.b * sizeof(double2), cudaMemcpyHostToDevice, c.s);
  k_axpby<<<nblocks(c.N * c.b), 256, 0, c.s>>>(d, x, ldx, d + c.b, y, ldy, c.N, c.b);
  // the host vectors may change right after: make the copies complete first
  return cudaStreamSynchronize(c.s) == cudaSuccess ? FIO_OK : FIO_ECUDA;
}

inline double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
inline double2 cmulh(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// preconditioner / inner correction in precision `prec`: y = G-dot K-dot* x (which = 3) or
// G-dot x (which = 2); x, y FP64 with ld = N
int precond(Ctx& c, Work& w, int which, const double2* x, double2* y, int prec) {
  if (prec == FIO_P64) return fio_apply_internal(c.op, which, x, y, c.N, c.b, FIO_P64, c.s);
  const long long n = c.N * c.b;
  k_to32<<<nblocks(n), 256, 0, c.s>>>(x, w.v32[0], n);
  int rc = fio_apply_internal(c.op, which, w.v32[0], w.v32[1], c.N, c.b, prec, c.s);
  if (rc) return rc;
  cudaMemsetAsync(y, 0, n * sizeof(double2), c.s);
  k_add32<<<nblocks(n), 256, 0, c.s>>>(w.v32[1], y, c.N, c.N, c.b);
  return cudaGetLastError() == cudaSuccess ? FIO_OK : FIO_ECUDA;
}

// s = u - K-dot f   (s, tmp: ld N; u, f: ld), K-dot in the outer precision; when f is known to
// be zero, s = u without an apply
int residual(Ctx& c, const double2* u, long long ld, const double2* f, double2* s) {
  if (c.f_zero) {
    c.f_zero = false;
    return cudaMemcpy2DAsync(s, c.N * sizeof(double2), u, ld * sizeof(double2), c.N * sizeof(double2), c.b,
                             cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
               ? FIO_OK
               : FIO_ECUDA;
  }
  int rc = fio_apply_internal(c.rop, 0, f, s, ld, c.b, c.outer, c.s);
  if (rc) return rc;
  std::vector<double2> one(c.b, make_double2(1, 0)), mone(c.b, make_double2(-1, 0));
  // s holds K f with ld = ld; bring it to ld N: s = u - s
  if (ld != c.N) return FIO_EINVAL;
  return axpby(c, one, u, ld, mone, s, c.N);
}

}  // namespace

void fio_solver_free(fio_op op) {
  if (op && op->solver) {
    cudaFree(op->solver);
    op->solver = nullptr;
    op->solver_bytes = 0;
  }
}

extern "C" int fio_solve(fio_op op, const void* uv, void* fv, int64_t ld, int b, int dtype,
                         const fio_solve_opts* opts, fio_solve_info* info, void* stream) {
  if (!op || !opts || b < 0 || dtype != FIO_C128 || ld != op->N) return FIO_EINVAL;
  if (b > 0 && (!uv || !fv || uv == fv)) return FIO_EINVAL;
  if (opts->method < FIO_DIRECT || opts->method > FIO_IR) return FIO_EINVAL;
  if (opts->inner < FIO_P64 || opts->inner > FIO_PTF32X3) return FIO_EINVAL;
  if (opts->inner != FIO_P64 && !op->arena32) return FIO_EINVAL;
  if (is_tc_precision(opts->inner) && !op->arena_tc) return FIO_EINVAL;
  if (opts->outer != FIO_P64 && opts->outer != FIO_PDF) return FIO_EINVAL;
  if (opts->outer == FIO_PDF && !op->arena_df) return FIO_EINVAL;
  fio_op rop = opts->residual_op ? opts->residual_op : op;
  if (rop != op) {
    if (opts->method != FIO_IR && opts->method != FIO_DIRECT) return FIO_EINVAL;
    if (rop->d != op->d || rop->n != op->n || rop->N != op->N) return FIO_EINVAL;
    if (opts->outer == FIO_PDF ? !rop->arena_df : !rop->arena) return FIO_EINVAL;
  }
  if (op->n_root == 0) return FIO_ENOTSUP;
  if (b == 0) return FIO_OK;
  const int maxit = opts->maxit > 0 ? opts->maxit : 100;
  const int restart = opts->method == FIO_GMRES ? (opts->restart > 0 ? opts->restart : 20) : 1;
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  int rc = get_work(op, b, restart, &w);
  if (rc) return rc;
  Ctx c{op, rop, op->N, b, s, w.sc};
  c.outer = opts->outer;
  const double2* u = (const double2*)uv;
  double2* f = (double2*)fv;
  const long long N = op->N;
  std::vector<double2> tmp;
  rc = dots(c, u, N, u, N, w.sc + 2 * b, &tmp);
  if (rc) return rc;
  std::vector<double> unorm(b);
  for (int j = 0; j < b; ++j) unorm[j] = sqrt(tmp[j].x) > 0 ? sqrt(tmp[j].x) : 1.0;
  if (opts->method != FIO_DIRECT) {  // a zero initial guess needs no apply for its residual
    rc = dots(c, f, N, f, N, w.sc + 2 * b, &tmp);
    if (rc) return rc;
    c.f_zero = true;
    for (int j = 0; j < b; ++j) c.f_zero = c.f_zero && tmp[j].x == 0.0;
  }
  std::vector<double> relres(b, 1.0);
  std::vector<int> iters(b, 0);
  std::vector<char> done(b, 0);
  const double tol = opts->tol;

  auto all_done = [&]() {
    for (int j = 0; j < b; ++j)
      if (!done[j]) return false;
    return true;
  };

  double2* S = w.v[0];  // true residual u - K f
  if (opts->method == FIO_DIRECT) {
    rc = precond(c, w, 3, u, f, opts->inner);
    if (rc) return rc;
    rc = residual(c, u, N, f, S);
    if (rc) return rc;
    rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
    if (rc) return rc;
    for (int j = 0; j < b; ++j) relres[j] = sqrt(tmp[j].x) / unorm[j];
  } else if (opts->method == FIO_IR) {
    double2* D = w.v[1];
    for (int it = 0;; ++it) {
      rc = residual(c, u, N, f, S);
      if (rc) return rc;
      rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
      if (rc) return rc;
      for (int j = 0; j < b; ++j) {
        relres[j] = sqrt(tmp[j].x) / unorm[j];
        if (!done[j]) iters[j] = it;
        if (relres[j] <= tol) done[j] = 1;
      }
      if (all_done() || it >= maxit) break;
      rc = precond(c, w, 3, S, D, opts->inner);
      if (rc) return rc;
      std::vector<double2> al(b), one(b, make_double2(1, 0));
      for (int j = 0; j < b; ++j) al[j] = done[j] ? make_double2(0, 0) : make_double2(1, 0);
      rc = axpby(c, al, D, N, one, f, N);
      if (rc) return rc;
    }
  } else if (opts->method == FIO_PCG) {
    double2 *Rn = w.v[1], *Z = w.v[2], *P = w.v[3], *Wv = w.v[4], *Q = w.v[5];
    rc = residual(c, u, N, f, S);
    if (rc) return rc;
    rc = fio_apply_internal(op, 1, S, Rn, N, b, FIO_P64, s);  // r = K* s
    if (rc) return rc;
    rc = precond(c, w, 2, Rn, Z, opts->inner);
    if (rc) return rc;
    std::vector<double2> zero(b, make_double2(0, 0)), one(b, make_double2(1, 0));
    rc = axpby(c, one, Z, N, zero, P, N);
    if (rc) return rc;
    std::vector<double2> rho;
    rc = dots(c, Rn, N, Z, N, w.sc + 2 * b, &rho);
    if (rc) return rc;
    rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
    if (rc) return rc;
    for (int j = 0; j < b; ++j) {
      relres[j] = sqrt(tmp[j].x) / unorm[j];
      if (relres[j] <= tol) done[j] = 1;
    }
    for (int it = 1; it <= maxit && !all_done(); ++it) {
      rc = fio_apply_internal(op, 0, P, Wv, N, b, FIO_P64, s);  // w = K p
      if (rc) return rc;
      rc = fio_apply_internal(op, 1, Wv, Q, N, b, FIO_P64, s);  // q = K* w
      if (rc) return rc;
      std::vector<double2> ww;
      rc = dots(c, Wv, N, Wv, N, w.sc + 2 * b, &ww);
      if (rc) return rc;
      std::vector<double2> al(b), mal(b);
      for (int j = 0; j < b; ++j) {
        const double2 a = (done[j] || ww[j].x == 0) ? make_double2(0, 0) : make_double2(rho[j].x / ww[j].x, rho[j].y / ww[j].x);
        al[j] = a;
        mal[j] = make_double2(-a.x, -a.y);
      }
      if ((rc = axpby(c, al, P, N, one, f, N))) return rc;
      if ((rc = axpby(c, mal, Wv, N, one, S, N))) return rc;
      if ((rc = axpby(c, mal, Q, N, one, Rn, N))) return rc;
      rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
      if (rc) return rc;
      for (int j = 0; j < b; ++j) {
        if (done[j]) continue;
        iters[j] = it;
        relres[j] = sqrt(tmp[j].x) / unorm[j];
        if (relres[j] <= tol) done[j] = 1;
      }
      if (all_done()) break;
      rc = precond(c, w, 2, Rn, Z, opts->inner);
      if (rc) return rc;
      std::vector<double2> rho_new;
      rc = dots(c, Rn, N, Z, N, w.sc + 2 * b, &rho_new);
      if (rc) return rc;
      std::vector<double2> be(b);
      for (int j = 0; j < b; ++j) be[j] = done[j] ? make_double2(0, 0) : cdiv(rho_new[j], rho[j]);
      if ((rc = axpby(c, one, Z, N, be, P, N))) return rc;
      rho = rho_new;
    }
  } else {  // GMRES, right preconditioned with P = G-dot K-dot*
    const long long vs = N * b;  // stride between basis vectors
    double2* V = w.basis;
    double2* Zt = w.v[1];
    double2* Wv = w.v[2];
    int total_it = 0;
    while (!all_done() && total_it < maxit) {
      rc = residual(c, u, N, f, S);
      if (rc) return rc;
      rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
      if (rc) return rc;
      std::vector<double> beta(b);
      for (int j = 0; j < b; ++j) {
        beta[j] = sqrt(tmp[j].x);
        relres[j] = beta[j] / unorm[j];
        if (relres[j] <= tol) done[j] = 1;
      }
      if (all_done()) break;
      std::vector<double2> inv(b), zero(b, make_double2(0, 0));
      for (int j = 0; j < b; ++j) inv[j] = make_double2(beta[j] > 0 ? 1.0 / beta[j] : 0.0, 0);
      if ((rc = axpby(c, inv, S, N, zero, V, N))) return rc;
      // per-column Hessenberg (column-major (restart+1) x restart), Givens, rhs g
      std::vector<std::vector<double2>> H(b, std::vector<double2>((size_t)(restart + 1) * restart));
      std::vector<std::vector<double2>> cs(b, std::vector<double2>(restart)), sn(b, std::vector<double2>(restart));
      std::vector<std::vector<double2>> g(b, std::vector<double2>(restart + 1, make_double2(0, 0)));
      for (int j = 0; j < b; ++j) g[j][0] = make_double2(beta[j], 0);
      int k = 0;
      std::vector<char> active(b);
      for (int j = 0; j < b; ++j) active[j] = !done[j];
      for (; k < restart && total_it < maxit; ++k) {
        // w = K P v_k
        rc = precond(c, w, 3, V + (long long)k * vs, Zt, opts->inner);
        if (rc) return rc;
        rc = fio_apply_internal(op, 0, Zt, Wv, N, b, FIO_P64, s);
        if (rc) return rc;
        std::vector<double2> h1((size_t)(k + 1) * b), h2((size_t)(k + 1) * b);
        for (int pass = 0; pass < 2; ++pass) {
          dim3 grid(k + 1, b);
          k_basisdot<<<grid, kRedThreads, 0, s>>>(V, vs, Wv, N, b, k + 1, w.Hd);
          k_basis_sub<<<nblocks(N * b), 256, 0, s>>>(V, vs, Wv, N, b, k + 1, w.Hd);
          auto& dst = pass ? h2 : h1;
          if (cudaMemcpyAsync(dst.data(), w.Hd, (size_t)(k + 1) * b * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return FIO_ECUDA;
        }
        rc = dots(c, Wv, N, Wv, N, w.sc + 2 * b, &tmp);
        if (rc) return rc;
        ++total_it;
        std::vector<double2> inv2(b);
        for (int j = 0; j < b; ++j) {
          double2* Hj = H[j].data() + (size_t)k * (restart + 1);
          for (int i = 0; i <= k; ++i) {
            const double2 a = h1[i + (size_t)(k + 1) * j], bb = h2[i + (size_t)(k + 1) * j];
            Hj[i] = make_double2(a.x + bb.x, a.y + bb.y);
          }
          const double hn = sqrt(tmp[j].x);
          Hj[k + 1] = make_double2(hn, 0);
          inv2[j] = make_double2(hn > 0 ? 1.0 / hn : 0.0, 0);
          if (!active[j]) continue;
          for (int i = 0; i < k; ++i) {  // apply previous rotations
            const double2 a = Hj[i], bb = Hj[i + 1];
            const double2 ci = cs[j][i], si = sn[j][i];
            // [c s; -conj(s) c] with c real
            Hj[i] = make_double2(ci.x * a.x + (si.x * bb.x - si.y * bb.y), ci.x * a.y + (si.x * bb.y + si.y * bb.x));
            Hj[i + 1] = make_double2(-(si.x * a.x + si.y * a.y) + ci.x * bb.x, -(si.x * a.y - si.y * a.x) + ci.x * bb.y);
          }
          // rotation G = [c s; -conj(s) c], c = |a|/nu, s = (a/|a|) h/nu, zeroes h = H[k+1][k]
          const double2 a = Hj[k];
          const double na = sqrt(cabs2(a)), nu = sqrt(cabs2(a) + hn * hn);
          double2 ci = make_double2(1, 0), si = make_double2(0, 0);
          if (nu > 0 && na == 0) {
            ci = make_double2(0, 0);
            si = make_double2(1, 0);
          } else if (nu > 0) {
            ci = make_double2(na / nu, 0);
            si = make_double2(a.x / na * hn / nu, a.y / na * hn / nu);
          }
          cs[j][k] = ci;
          sn[j][k] = si;
          Hj[k] = make_double2(ci.x * a.x + si.x * hn, ci.x * a.y + si.y * hn);
          Hj[k + 1] = make_double2(0, 0);
          const double2 gk = g[j][k];
          g[j][k] = make_double2(ci.x * gk.x, ci.x * gk.y);
          g[j][k + 1] = make_double2(-(si.x * gk.x + si.y * gk.y), -(si.x * gk.y - si.y * gk.x));
          relres[j] = sqrt(cabs2(g[j][k + 1])) / unorm[j];
          iters[j] = total_it;
          if (relres[j] <= tol) active[j] = 0;
        }
        // v_{k+1} = w / ||w||
        std::vector<double2> zero2(b, make_double2(0, 0));
        if ((rc = axpby(c, inv2, Wv, N, zero2, V + (long long)(k + 1) * vs, N))) return rc;
        bool any = false;
        for (int j = 0; j < b; ++j) any = any || active[j];
        if (!any) {
          ++k;
          break;
        }
      }
      // y = H^{-1} g (upper triangular k x k per column); f += P (V y)
      std::vector<double2> coef((size_t)k * b, make_double2(0, 0));
      for (int j = 0; j < b; ++j) {
        if (done[j]) continue;
        std::vector<double2> y(k);
        for (int i = k - 1; i >= 0; --i) {
          double2 acc = g[j][i];
          for (int t = i + 1; t < k; ++t) {
            const double2 h = H[j][(size_t)t * (restart + 1) + i];
            const double2 p = cmulh(h, y[t]);
            acc.x -= p.x;
            acc.y -= p.y;
          }
          y[i] = cdiv(acc, H[j][(size_t)i * (restart + 1) + i]);
        }
        for (int i = 0; i < k; ++i) coef[i + (size_t)k * j] = y[i];
      }
      // Zt = V y  (reuse k_basis_sub with negated coefficients on a zeroed vector)
      for (auto& v : coef) v = make_double2(-v.x, -v.y);
      cudaMemsetAsync(Zt, 0, (size_t)N * b * sizeof(double2), s);
      cudaMemcpyAsync(w.Hd, coef.data(), coef.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
      if (k > 0) k_basis_sub<<<nblocks(N * b), 256, 0, s>>>(V, vs, Zt, N, b, k, w.Hd);
      rc = precond(c, w, 3, Zt, Wv, opts->inner);
      if (rc) return rc;
      std::vector<double2> one(b, make_double2(1, 0));
      if ((rc = axpby(c, one, Wv, N, one, f, N))) return rc;
    }
    // final true residual
    rc = residual(c, u, N, f, S);
    if (rc) return rc;
    rc = dots(c, S, N, S, N, w.sc + 2 * b, &tmp);
    if (rc) return rc;
    for (int j = 0; j < b; ++j) {
      relres[j] = sqrt(tmp[j].x) / unorm[j];
      if (relres[j] <= tol) done[j] = 1;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return FIO_ECUDA;
  if (fio_tc_timeout_reset() > 0) return FIO_ETIMEOUT;
  bool conv = true;
  for (int j = 0; j < b; ++j) {
    const bool ok = relres[j] <= tol || opts->method == FIO_DIRECT;
    conv = conv && ok;
    if (info) {
      info[j].iters = opts->method == FIO_DIRECT ? 0 : iters[j];
      info[j].relres = relres[j];
      info[j].status = ok ? FIO_OK : FIO_ENOCONV;
    }
  }
  return conv ? FIO_OK : FIO_ENOCONV;
}

// refine.cu — FP64 refinement around an FP32 factor (mixed precision).
//
// The factor L32 is computed and stored in FP32 (the FP32 FMA pipe is ~60x the FP64 one on
// GB300); accuracy is won back in FP64 by conjugate gradients on A x = b preconditioned with
// M = L32 L32^T. The residual b - A x, the solution and every inner product stay in FP64; only
// the preconditioner solves run in FP32. When M is close to A (kappa(A) u32 << 1) the first
// iterate is already the FP32 solution and each further iteration gains about -log10(kappa u32)
// digits, as in classic iterative refinement; unlike plain refinement, CG also converges when the
// FP32 factor is poor, because M stays symmetric positive definite.
//
// Everything runs in the permuted space of the factor: b~ = P b, C = P A P^T (held as a full
// CSR whose values are gathered from A's entries), x = P^T x~ at the end. Reductions are
// deterministic (fixed partition, two passes). Convergence is judged per right-hand side by the
// normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kernels.h"
#include "refine.h"

namespace sym {
namespace {

constexpr int RT = 256;        // threads per block of the vector kernels
constexpr int RBLOCKS = 304;   // blocks per column of the first reduction pass (2 per SM)

// out = B - C X (minus = true) or out = C X, column by column; thread per row.
__global__ void k_spmv(const int64_t *__restrict__ cp, const int32_t *__restrict__ ci,
                       const int64_t *__restrict__ cmap, const double *__restrict__ Ax,
                       const double *__restrict__ X, const double *__restrict__ B, double *__restrict__ out,
                       int64_t n, int nrhs, bool minus) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p0 = cp[i], p1 = cp[i + 1];
  for (int c = 0; c < nrhs; ++c) {
    const double *x = X + (int64_t)c * n;
    double s = 0.0;
    for (int64_t p = p0; p < p1; ++p) s = fma(Ax[cmap[p]], x[ci[p]], s);
    out[(int64_t)c * n + i] = minus ? B[(int64_t)c * n + i] - s : s;
  }
}

// ||A||_inf of C: per-row absolute sums (first pass writes them, the max pass reduces).
__global__ void k_rowabs(const int64_t *__restrict__ cp, const int64_t *__restrict__ cmap,
                         const double *__restrict__ Ax, double *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t p = cp[i]; p < cp[i + 1]; ++p) s += fabs(Ax[cmap[p]]);
  out[i] = s;
}

// First reduction pass: block b of column c covers a fixed slice of rows. mode 0: sum of
// a*b; mode 1: max |a|.
__global__ void k_reduce1(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ part,
                          int64_t n, int mode) {
  __shared__ double sh[RT];
  const int c = blockIdx.y;
  const int64_t chunk = (n + RBLOCKS - 1) / RBLOCKS;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  const double *ac = a + (int64_t)c * n;
  const double *bc = b ? b + (int64_t)c * n : nullptr;
  double v = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += RT) v = mode == 0 ? fma(ac[i], bc[i], v) : fmax(v, fabs(ac[i]));
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = mode == 0 ? sh[threadIdx.x] + sh[threadIdx.x + s] : fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)c * RBLOCKS + blockIdx.x] = sh[0];
}

// Second pass: one block per column folds its RBLOCKS partial results.
__global__ void k_reduce2(const double *__restrict__ part, double *__restrict__ out, int mode) {
  __shared__ double sh[RT];
  const int c = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < RBLOCKS; i += RT) {
    const double x = part[(int64_t)c * RBLOCKS + i];
    v = mode == 0 ? v + x : fmax(v, x);
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = mode == 0 ? sh[threadIdx.x] + sh[threadIdx.x + s] : fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// Per-column CG scalars. alpha = rho / (p^T q); beta = rho_new / rho (then rho = rho_new).
__global__ void k_alpha(const double *__restrict__ rho, const double *__restrict__ pq, double *__restrict__ alpha, int nrhs) {
  const int c = threadIdx.x;
  if (c < nrhs) alpha[c] = (pq[c] > 0.0 && rho[c] > 0.0) ? rho[c] / pq[c] : 0.0;
}
__global__ void k_beta(double *__restrict__ rho, const double *__restrict__ rho_new, double *__restrict__ beta, int nrhs) {
  const int c = threadIdx.x;
  if (c < nrhs) {
    beta[c] = rho[c] > 0.0 ? rho_new[c] / rho[c] : 0.0;
    rho[c] = rho_new[c];
  }
}

// x += alpha p; r -= alpha q.
__global__ void k_update_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ q, const double *__restrict__ alpha, int64_t n, int nrhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const double a = alpha[i / n];
  x[i] = fma(a, p[i], x[i]);
  r[i] = fma(-a, q[i], r[i]);
}
// p = z + beta p (beta == nullptr: p = z).
__global__ void k_update_p(double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ beta,
                           int64_t n, int nrhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  p[i] = beta ? fma(beta[i / n], p[i], z[i]) : z[i];
}
__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) b[i] = (float)a[i];
}
__global__ void k_to_double(const float *__restrict__ a, double *__restrict__ b, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) b[i] = (double)a[i];
}
__global__ void k_fill(double *__restrict__ a, double v, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) a[i] = v;
}

inline unsigned blocks(int64_t count) { return (unsigned)((count + RT - 1) / RT); }

}  // namespace

void precond_graph_reset(PrecondGraph &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g = PrecondGraph();
}

int64_t refine_work_doubles(int64_t n, int nrhs) {
  // x, r, z, p, q, b~ (n x nrhs each) + float block (half) + partials + 8 scalar arrays
  return 6 * n * nrhs + (n * nrhs + 1) / 2 + (int64_t)RBLOCKS * nrhs + 8 * 64 + n;
}

cudaError_t refine_anorm(const RefineCtx &c, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  double *rowabs = c.anorm_work;  // n doubles of scratch
  double *part = c.anorm_work + c.n;
  k_rowabs<<<blocks(c.n), RT, 0, st>>>(c.cp, c.cmap, c.Ax, rowabs, c.n);
  k_reduce1<<<dim3(RBLOCKS, 1), RT, 0, st>>>(rowabs, nullptr, part, c.n, 1);
  k_reduce2<<<1, RT, 0, st>>>(part, c.anorm, 1);
  return cudaGetLastError();
}

int refine_solve(const RefineCtx &c, int nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                 double tol, int max_iter, double *host_eta, RefineResult *res, cudaStream_t st) {
  res->iterations = 0;
  res->backward_error = 0.0;
  res->converged = true;
  const int64_t n = c.n;
  if (n == 0 || nrhs == 0) return 0;
  const int64_t nn = n * nrhs;
  double *x = c.work, *r = x + nn, *z = r + nn, *p = z + nn, *q = p + nn, *bt = q + nn;
  float *yf = reinterpret_cast<float *>(bt + nn);
  double *part = bt + nn + (nn + 1) / 2;
  double *sc = part + (int64_t)RBLOCKS * nrhs;  // scalar arrays, 64 entries each
  double *rho = sc, *rho_new = sc + 64, *pq = sc + 128, *alpha = sc + 192, *beta = sc + 256,
         *rmax = sc + 320, *xmax = sc + 384, *bmax = sc + 448;
  auto reduce = [&](const double *a, const double *b, double *out, int mode) {
    k_reduce1<<<dim3(RBLOCKS, nrhs), RT, 0, st>>>(a, b, part, n, mode);
    k_reduce2<<<nrhs, RT, 0, st>>>(part, out, mode);
  };
  auto enqueue_precond = [&](const double *in, double *out, cudaStream_t s) -> cudaError_t {
    k_to_float<<<blocks(nn), RT, 0, s>>>(in, yf, nn);
    cudaError_t e = run_sweeps<float, float>(*c.dp, *c.fwd, *c.bwd, c.Lf, c.Lfinv, nrhs, yf, s, nullptr);
    if (e != cudaSuccess) return e;
    k_to_double<<<blocks(nn), RT, 0, s>>>(yf, out, nn);
    return cudaGetLastError();
  };
  auto precond = [&](const double *in, double *out) -> cudaError_t {
    if (!c.pgraph || !c.capture) return enqueue_precond(in, out, st);
    PrecondGraph &g = *c.pgraph;
    if (!(g.exec && g.key[0] == in && g.key[1] == out && g.key[2] == yf && g.key[3] == c.Lf && g.nrhs == nrhs)) {
      precond_graph_reset(g);
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c.capture, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      const cudaError_t e1 = enqueue_precond(in, out, c.capture);
      const cudaError_t e2 = cudaStreamEndCapture(c.capture, &gr);
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return e1 != cudaSuccess ? e1 : e2;
      }
      e = cudaGraphInstantiate(&g.exec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        g.exec = nullptr;
        return e;
      }
      g.key[0] = in;
      g.key[1] = out;
      g.key[2] = yf;
      g.key[3] = c.Lf;
      g.nrhs = nrhs;
    }
    return cudaGraphLaunch(g.exec, st);
  };
  // b~ = P b; x = 0; r = b~
  if (permute_in<double>(*c.dp, nrhs, B, ldb, bt, st) != cudaSuccess) return -1;
  k_fill<<<blocks(nn), RT, 0, st>>>(x, 0.0, nn);
  cudaMemcpyAsync(r, bt, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st);
  reduce(bt, nullptr, bmax, 1);
  auto restart = [&]() -> cudaError_t {
    cudaError_t e = precond(r, z);
    if (e != cudaSuccess) return e;
    k_update_p<<<blocks(nn), RT, 0, st>>>(p, z, nullptr, n, nrhs);
    reduce(r, z, rho, 0);
    return cudaGetLastError();
  };
  if (restart() != cudaSuccess) return -1;
  std::vector<double> hb(nrhs);
  double anorm = 0.0;
  bool have_norms = false;
  int it = 0;
  // host_eta layout: [0,64) ||r||_inf, [64,128) ||x||_inf, [128,192) ||b||_inf, [192] ||A||_inf
  auto eta_worst = [&]() {
    double worst = 0.0;
    for (int k = 0; k < nrhs; ++k) {
      const double den = anorm * host_eta[64 + k] + hb[k];
      const double eta = den > 0 ? host_eta[k] / den : 0.0;
      worst = eta > worst ? eta : worst;
    }
    return worst;
  };
  while (true) {
    // q = C p; alpha = rho / p^T q; x += alpha p; r -= alpha q
    k_spmv<<<blocks(n), RT, 0, st>>>(c.cp, c.ci, c.cmap, c.Ax, p, nullptr, q, n, nrhs, false);
    reduce(p, q, pq, 0);
    k_alpha<<<1, 64, 0, st>>>(rho, pq, alpha, nrhs);
    k_update_xr<<<blocks(nn), RT, 0, st>>>(x, r, p, q, alpha, n, nrhs);
    ++it;
    reduce(r, nullptr, rmax, 1);
    reduce(x, nullptr, xmax, 1);
    cudaMemcpyAsync(host_eta, rmax, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(host_eta + 64, xmax, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
    if (!have_norms) {
      cudaMemcpyAsync(host_eta + 128, bmax, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(host_eta + 192, c.anorm, sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    if (!have_norms) {
      for (int k = 0; k < nrhs; ++k) hb[k] = host_eta[128 + k];
      anorm = host_eta[192];
      have_norms = true;
    }
    res->backward_error = eta_worst();
    if (res->backward_error <= tol) {
      // Every claim of convergence is confirmed with the true residual r = b~ - C x.
      k_spmv<<<blocks(n), RT, 0, st>>>(c.cp, c.ci, c.cmap, c.Ax, x, bt, r, n, nrhs, true);
      reduce(r, nullptr, rmax, 1);
      cudaMemcpyAsync(host_eta, rmax, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
      res->backward_error = eta_worst();
      if (res->backward_error <= tol) break;
      if (it >= max_iter) {
        res->converged = false;
        break;
      }
      if (restart() != cudaSuccess) return -1;  // continue from the true residual
      continue;
    }
    if (it >= max_iter) {
      res->converged = false;
      break;
    }
    // z = M^-1 r; beta = rho_new / rho; p = z + beta p
    if (precond(r, z) != cudaSuccess) return -1;
    reduce(r, z, rho_new, 0);
    k_beta<<<1, 64, 0, st>>>(rho, rho_new, beta, nrhs);
    k_update_p<<<blocks(nn), RT, 0, st>>>(p, z, beta, n, nrhs);
  }
  res->iterations = it;
  if (permute_out<double>(*c.dp, nrhs, x, X, ldx, st) != cudaSuccess) return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sym

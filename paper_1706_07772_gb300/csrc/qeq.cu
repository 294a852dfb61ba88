// (e) QEq charge equilibration: two Jacobi-preconditioned CG solves on one H matrix.
//
// Paper: Sec. 3.3 "QEq": the Lagrange-multiplier form gives two systems with a common
// sparse H (H s = -chi, H t = -1), solved with a diagonally preconditioned CG from an
// extrapolated initial guess; the two systems are iterated concurrently (one pass over H
// for both vectors, merged reductions). Charges q = s - (sum s / sum t) t.
// H_ii = eta_i, H_ij = Tap(r) k_e / (r^3 + gamma_ij^-3)^(1/3) summed over images in range
// (its entries are written by the far-list pass).
//
// GPU form: one persistent cooperative kernel runs the whole solve. Per iteration:
//   A: u = H z (both systems in one read of H), p = z + beta p, w = u + beta w, p.w
//   B: x += alpha p, r -= alpha w, z = r / eta, r.z and r.r
// (w = H p is carried as H z + beta w, so H is read once per iteration.) Each phase ends
// in a grid barrier whose last-arriving block reduces the per-chunk partial dot products
// per replica in a fixed order (deterministic) and publishes alpha, beta and the
// convergence flags. Convergence per system and replica: ||r||_2 <= tol ||b||_2; a
// converged system freezes while the other continues. Barrier waits are bounded.
#include "reax_internal.cuh"

namespace {

constexpr int NQ = 8;          // partial sums per chunk
constexpr int NS = 16;         // scalars per replica
// scalar slots per replica
enum { S_RHO_S = 0, S_RHO_T, S_AL_S, S_AL_T, S_BE_S, S_BE_T, S_BB_S, S_BB_T, S_ACT_S, S_ACT_T, S_MU };

template <typename R>
struct CG {
  int n, nrep, nchunk, max_iter;
  double tol2;
  const int* type;
  const int* rep;
  const int* cnt;
  const int* col;
  const R* H;
  int cap;
  const int* cntn;                         // near part of each row
  const int* coln;
  const R* Hn;
  int capn;
  const double *eta, *chi, *ieta;          // per type (double); ieta = 1/eta
  double *xs, *xt, *rs, *rt, *zs, *zt, *ps, *pt, *ws, *wt;
  float *zsf, *ztf;                        // FP32 copies of z for the FP32-arithmetic SpMV
  double* q;
  float* qf;
  double* part;                            // [nchunk*NQ]
  double* red;                             // [nrep*NQ]
  double* scal;                            // [nrep*NS + 1]
  const int* chunk_lo;                     // [nchunk+1] rows
  const int* chunk_rep;                    // [nchunk]
  const int* rep_chunk;                    // [nrep+1] chunk ranges per replica
  int* iters;                              // [2*nrep]
  GridBar* bar;
  int* err;
};

// grid barrier; the last block to arrive runs `reduce` (whole block) before releasing
template <typename F>
__device__ bool barrier_reduce(GridBar* bar, int* err, F reduce) {
  __shared__ int s_last;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g = *((volatile unsigned*)&bar->gen);
    __threadfence();
    unsigned a = atomicAdd(&bar->arrive, 1u);
    s_last = (a == gridDim.x - 1);
    s_gen = g;
  }
  __syncthreads();
  bool ok = true;
  if (s_last) {
    __threadfence();
    reduce();
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      bar->arrive = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    }
  } else {
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (*((volatile unsigned*)&bar->gen) == s_gen) {
        if (++spins > BAR_SPIN_LIMIT) {
          atomicOr(err, ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
  }
  __syncthreads();
  if (*((volatile int*)err) & ERR_TIMEOUT) ok = false;
  return ok;
}

// last-block reduction of chunk partials into red[r*NQ+q]: one warp per replica, each
// lane sums whole chunks (all NQ slots, contiguous) in a fixed order, then the lanes are
// combined by a fixed butterfly (deterministic)
template <typename R>
__device__ void reduce_parts(const CG<R>& a, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = wid; r < a.nrep; r += nw) {
    double v[NQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = a.rep_chunk[r] + lane; c < a.rep_chunk[r + 1]; c += 32) {
      const double2* src = (const double2*)(a.part + (size_t)c * NQ);
#pragma unroll
      for (int q = 0; q < NQ / 2; ++q) {
        const double2 t = __ldcg(src + q);
        v[2 * q] += t.x;
        v[2 * q + 1] += t.y;
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
    if (lane < NQ) {
      double o = v[0];
#pragma unroll
      for (int q = 1; q < NQ; ++q) o = lane == q ? v[q] : o;
      red[r * NQ + lane] = o;
    }
  }
  __syncthreads();
}

// block-level partial sums of NQ values held by lane 0 of each warp (the lane that does
// the row's scalar work) -> part[chunk*NQ + q], summed over warps in a fixed order
__device__ __forceinline__ void block_partials(double* vals, double* part, int chunk) {
  __shared__ double sh[32][NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[wid][q] = vals[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += sh[w][threadIdx.x];
    part[chunk * NQ + threadIdx.x] = v;
  }
  __syncthreads();
}

// (H v)_i for the two systems, warp per row. FP64 path: FP64 products and sums. Mixed
// path: H and v in FP32, FP32 products and per-lane partial sums (about 13 terms per
// lane), lanes combined in FP64 -- FP64 work per row drops from 2 per entry to ~10.
template <typename R>
__device__ __forceinline__ void spmv_part(const int* cnt, const int* col, const R* H, int cap, int i, const double* vs,
                                          const double* vt, const float* vsf, const float* vtf, double& s1, double& t1) {
  const int lane = threadIdx.x & 31;
  const int row = i * cap, nf = cnt[i];
  if (sizeof(R) == 4) {
    // each lane takes 4 consecutive entries per pass (one int4 + one float4 load: rows start
    // at multiples of 32 entries, so 16-byte aligned), then 4 independent gathers of z
    float sf = 0.0f, tf = 0.0f;
    const int4* c4 = (const int4*)(col + row);
    const float4* h4 = (const float4*)((const float*)H + row);
    for (int k = 4 * lane; k < nf; k += 128) {
      const int4 cc = __ldg(c4 + (k >> 2));
      const float4 hh = __ldg(h4 + (k >> 2));
      const int jj[4] = {cc.x, cc.y, cc.z, cc.w};
      const float hv[4] = {hh.x, hh.y, hh.z, hh.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (k + u < nf) {
          sf = fmaf(hv[u], __ldcg(&vsf[jj[u]]), sf);
          tf = fmaf(hv[u], __ldcg(&vtf[jj[u]]), tf);
        }
      }
    }
    s1 += (double)warp_sumf(sf);       // FP32 row reduction (H itself is FP32 here)
    t1 += (double)warp_sumf(tf);
  } else {
    for (int k = lane; k < nf; k += 32) {
      const int j = col[row + k];
      const double h = (double)H[row + k];
      s1 += h * __ldcg(&vs[j]);
      t1 += h * __ldcg(&vt[j]);
    }
  }
}
template <typename R>
__device__ __forceinline__ void spmv_row(const CG<R>& a, int i, const double* vs, const double* vt, const float* vsf,
                                         const float* vtf, double& hs, double& ht) {
  double s1 = 0.0, t1 = 0.0;
  spmv_part<R>(a.cntn, a.coln, a.Hn, a.capn, i, vs, vt, vsf, vtf, s1, t1);
  spmv_part<R>(a.cnt, a.col, a.H, a.cap, i, vs, vt, vsf, vtf, s1, t1);
  if (sizeof(R) == 8) {
    s1 = warp_sum(s1);
    t1 = warp_sum(t1);
  }
  const double d = a.eta[a.type[i]];
  hs = s1 + d * __ldcg(&vs[i]);
  ht = t1 + d * __ldcg(&vt[i]);
}

__device__ __forceinline__ double ldS(const double* p) { return __ldcg(p); }

template <typename R>
__global__ void __launch_bounds__(1024, 1) k_cg(CG<R> a) {
  double* red = a.red;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* S = a.scal;
  // ---------------- init: r = b - H x, z = r/eta, p = w = 0 (x copied to FP32 first)
  for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x)
    for (int i = a.chunk_lo[c] + threadIdx.x; i < a.chunk_lo[c + 1]; i += blockDim.x) {
      a.zsf[i] = (float)a.xs[i];
      a.ztf[i] = (float)a.xt[i];
    }
  bool ok0 = barrier_reduce(a.bar, a.err, []() {});
  if (!ok0) return;
  for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x) {
    double v[NQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = a.chunk_lo[c] + wid; i < a.chunk_lo[c + 1]; i += nw) {
      double hs, ht;
      spmv_row(a, i, a.xs, a.xt, a.zsf, a.ztf, hs, ht);
      if (lane == 0) {
        const double bs = -a.chi[a.type[i]], bt = -1.0, e = a.eta[a.type[i]];
        const double rs = bs - hs, rt = bt - ht;
        a.rs[i] = rs; a.rt[i] = rt;
        a.zs[i] = rs / e; a.zt[i] = rt / e;
        a.ps[i] = 0; a.pt[i] = 0; a.ws[i] = 0; a.wt[i] = 0;
        v[0] += rs * rs / e; v[1] += rt * rt / e;   // r.z
        v[2] += rs * rs; v[3] += rt * rt;           // r.r
        v[4] += bs * bs; v[5] += bt * bt;           // b.b
      }
    }
    block_partials(v, a.part, c);
  }
  bool ok = barrier_reduce(a.bar, a.err, [&]() {
    reduce_parts(a, red);
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
      double* sr = S + r * NS;
      const double* rd = red + r * NQ;
      sr[S_RHO_S] = rd[0]; sr[S_RHO_T] = rd[1];
      sr[S_BB_S] = rd[4]; sr[S_BB_T] = rd[5];
      sr[S_BE_S] = 0; sr[S_BE_T] = 0;
      sr[S_ACT_S] = rd[2] > a.tol2 * rd[4] ? 1.0 : 0.0;
      sr[S_ACT_T] = rd[3] > a.tol2 * rd[5] ? 1.0 : 0.0;
      a.iters[2 * r] = 0; a.iters[2 * r + 1] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double act = 0;
      for (int r = 0; r < a.nrep; ++r) act += S[r * NS + S_ACT_S] + S[r * NS + S_ACT_T];
      S[a.nrep * NS] = act;
    }
  });
  // z in FP32 for the first iteration's SpMV: written only after every block has finished
  // the initial SpMV (which read x from the same buffer), published by one more barrier
  if (ok) {
    for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x)
      for (int i = a.chunk_lo[c] + threadIdx.x; i < a.chunk_lo[c + 1]; i += blockDim.x) {
        a.zsf[i] = (float)a.zs[i];
        a.ztf[i] = (float)a.zt[i];
      }
    ok = barrier_reduce(a.bar, a.err, []() {});
  }
  int it = 0;
  while (ok && ldS(&S[a.nrep * NS]) > 0.0 && it < a.max_iter) {
    ++it;
    // ---------------- A: u = H z; p = z + beta p; w = u + beta w; p.w
    for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x) {
      const double* sr = S + a.chunk_rep[c] * NS;
      const bool as = ldS(sr + S_ACT_S) > 0, at = ldS(sr + S_ACT_T) > 0;
      const double bes = ldS(sr + S_BE_S), bet = ldS(sr + S_BE_T);
      double v[NQ] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int i = a.chunk_lo[c] + wid; i < a.chunk_lo[c + 1]; i += nw) {
        double us, ut;
        spmv_row(a, i, a.zs, a.zt, a.zsf, a.ztf, us, ut);
        if (lane == 0) {
          if (as) {
            const double p = a.zs[i] + bes * a.ps[i], w = us + bes * a.ws[i];
            a.ps[i] = p; a.ws[i] = w; v[0] += p * w;
          }
          if (at) {
            const double p = a.zt[i] + bet * a.pt[i], w = ut + bet * a.wt[i];
            a.pt[i] = p; a.wt[i] = w; v[1] += p * w;
          }
        }
      }
      block_partials(v, a.part, c);
    }
    ok = barrier_reduce(a.bar, a.err, [&]() {
      reduce_parts(a, red);
      for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
        double* sr = S + r * NS;
        sr[S_AL_S] = sr[S_ACT_S] > 0 ? sr[S_RHO_S] / red[r * NQ + 0] : 0.0;
        sr[S_AL_T] = sr[S_ACT_T] > 0 ? sr[S_RHO_T] / red[r * NQ + 1] : 0.0;
      }
    });
    if (!ok) break;
    // ---------------- B: x += alpha p; r -= alpha w; z = r / eta; r.z, r.r
    for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x) {
      const double* sr = S + a.chunk_rep[c] * NS;
      const bool as = ldS(sr + S_ACT_S) > 0, at = ldS(sr + S_ACT_T) > 0;
      const double als = ldS(sr + S_AL_S), alt = ldS(sr + S_AL_T);
      double v[NQ] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int i = a.chunk_lo[c] + wid; i < a.chunk_lo[c + 1]; i += nw) {
        if (lane != 0) continue;
        const double ie = a.ieta[a.type[i]];
        if (as) {
          a.xs[i] += als * a.ps[i];
          const double r = a.rs[i] - als * a.ws[i];
          const double z = r * ie;
          a.rs[i] = r; a.zs[i] = z; a.zsf[i] = (float)z;
          v[0] += r * z; v[2] += r * r;
        }
        if (at) {
          a.xt[i] += alt * a.pt[i];
          const double r = a.rt[i] - alt * a.wt[i];
          const double z = r * ie;
          a.rt[i] = r; a.zt[i] = z; a.ztf[i] = (float)z;
          v[1] += r * z; v[3] += r * r;
        }
      }
      block_partials(v, a.part, c);
    }
    ok = barrier_reduce(a.bar, a.err, [&]() {
      reduce_parts(a, red);
      for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
        double* sr = S + r * NS;
        if (sr[S_ACT_S] > 0) {
          a.iters[2 * r] += 1;
          sr[S_BE_S] = red[r * NQ + 0] / sr[S_RHO_S];
          sr[S_RHO_S] = red[r * NQ + 0];
          if (!(red[r * NQ + 2] > a.tol2 * sr[S_BB_S])) sr[S_ACT_S] = 0.0;
        }
        if (sr[S_ACT_T] > 0) {
          a.iters[2 * r + 1] += 1;
          sr[S_BE_T] = red[r * NQ + 1] / sr[S_RHO_T];
          sr[S_RHO_T] = red[r * NQ + 1];
          if (!(red[r * NQ + 3] > a.tol2 * sr[S_BB_T])) sr[S_ACT_T] = 0.0;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double act = 0;
        for (int r = 0; r < a.nrep; ++r) act += S[r * NS + S_ACT_S] + S[r * NS + S_ACT_T];
        S[a.nrep * NS] = act;
      }
    });
  }
  if (ok && ldS(&S[a.nrep * NS]) > 0.0 && blockIdx.x == 0 && threadIdx.x == 0)
    atomicOr(a.err, ERR_CG);
  if (!ok) return;
  // ---------------- charges: mu = sum s / sum t per replica, q = s - mu t
  for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x) {
    double v[NQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = a.chunk_lo[c] + wid; i < a.chunk_lo[c + 1]; i += nw) {
      if (lane != 0) continue;
      v[0] += a.xs[i];
      v[1] += a.xt[i];
    }
    block_partials(v, a.part, c);
  }
  ok = barrier_reduce(a.bar, a.err, [&]() {
    reduce_parts(a, red);
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) S[r * NS + S_MU] = red[r * NQ + 0] / red[r * NQ + 1];
  });
  if (!ok) return;
  for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x) {
    const double mu = ldS(&S[a.chunk_rep[c] * NS + S_MU]);
    for (int i = a.chunk_lo[c] + threadIdx.x; i < a.chunk_lo[c + 1]; i += blockDim.x) {
      const double qi = a.xs[i] - mu * a.xt[i];
      a.q[i] = qi;
      a.qf[i] = (float)qi;
    }
  }
}

// initial guess: Lagrange extrapolation of the solution history (cubic for s from 4
// points, quadratic for t from 3; lower order while the history is short; 0 without one)
__global__ void k_warm(int n, int nh, double* xs, double* xt, const double* h0s, const double* h1s,
                       const double* h2s, const double* h3s, const double* h0t, const double* h1t,
                       const double* h2t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0, t = 0;
  if (nh >= 4) s = 4 * h0s[i] - 6 * h1s[i] + 4 * h2s[i] - h3s[i];
  else if (nh == 3) s = 3 * h0s[i] - 3 * h1s[i] + h2s[i];
  else if (nh == 2) s = 2 * h0s[i] - h1s[i];
  else if (nh == 1) s = h0s[i];
  if (nh >= 3) t = 3 * h0t[i] - 3 * h1t[i] + h2t[i];
  else if (nh == 2) t = 2 * h0t[i] - h1t[i];
  else if (nh == 1) t = h0t[i];
  xs[i] = s;
  xt[i] = t;
}

}  // namespace

namespace rx {

template <typename R>
int qeq_solve(const Launch& L, Sys s, FarList f, QeqState& Q, const DParams<R>* P, const double* chi,
              const double* eta, double tol, int max_iter, int warm) {
  (void)P;
  const int nh = warm == REAXFF_WARM_EXTRAP ? Q.nhist : 0;
  k_warm<<<(s.n + 255) / 256, 256, 0, L.st>>>(s.n, nh, Q.s, Q.t, Q.hist_s + 0 * (size_t)s.n,
                                              Q.hist_s + 1 * (size_t)s.n, Q.hist_s + 2 * (size_t)s.n,
                                              Q.hist_s + 3 * (size_t)s.n, Q.hist_t + 0 * (size_t)s.n,
                                              Q.hist_t + 1 * (size_t)s.n, Q.hist_t + 2 * (size_t)s.n);
  CG<R> a;
  a.n = s.n; a.nrep = s.nrep; a.nchunk = Q.nchunk; a.max_iter = max_iter;
  a.tol2 = tol * tol;
  a.type = s.type; a.rep = s.rep;
  a.cnt = f.cnt; a.col = f.j; a.H = (const R*)f.H; a.cap = f.cap;
  a.cntn = f.cntn; a.coln = f.jn; a.Hn = (const R*)f.Hn; a.capn = f.capn;
  a.eta = eta; a.chi = chi;
  a.xs = Q.s; a.xt = Q.t; a.rs = Q.r_s; a.rt = Q.r_t; a.zs = Q.z_s; a.zt = Q.z_t;
  a.ps = Q.p_s; a.pt = Q.p_t; a.ws = Q.w_s; a.wt = Q.w_t;
  a.zsf = Q.zf_s; a.ztf = Q.zf_t;
  a.q = s.q; a.qf = s.qf; a.part = Q.part; a.red = Q.red; a.scal = Q.scal;
  a.ieta = Q.ieta;
  a.chunk_lo = Q.chunk_lo; a.chunk_rep = Q.chunk_rep; a.rep_chunk = Q.rep_chunk;
  a.iters = Q.iters; a.bar = Q.bar; a.err = s.err;
  cudaMemsetAsync(Q.bar, 0, sizeof(GridBar), L.st);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_cg<R>, dim3(Q.grid), dim3(1024), args, 0, L.st);
  *L.count += 2;
  return e == cudaSuccess ? 0 : -1;
}

// shift the history: newest solution becomes h0 (pointer rotation, one copy)
void qeq_push_history(const Launch& L, int n, QeqState& Q) {
  // rotate slots 3 <- 2 <- 1 <- 0 by copying (4 small device copies)
  cudaMemcpyAsync(Q.hist_s + 3 * (size_t)n, Q.hist_s + 2 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_s + 2 * (size_t)n, Q.hist_s + 1 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_s + 1 * (size_t)n, Q.hist_s + 0 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_s + 0 * (size_t)n, Q.s, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_t + 2 * (size_t)n, Q.hist_t + 1 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_t + 1 * (size_t)n, Q.hist_t + 0 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  cudaMemcpyAsync(Q.hist_t + 0 * (size_t)n, Q.t, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st);
  Q.nhist = Q.nhist < 4 ? Q.nhist + 1 : 4;
}

int qeq_grid_size(int nsm) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_cg<double>, 1024, 0);
  int per_f = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, (const void*)k_cg<float>, 1024, 0);
  if (per_f < per) per = per_f;
  if (per < 1) per = 1;
  return nsm * per;
}

template int qeq_solve<double>(const Launch&, Sys, FarList, QeqState&, const DParams<double>*, const double*,
                               const double*, double, int, int);
template int qeq_solve<float>(const Launch&, Sys, FarList, QeqState&, const DParams<float>*, const double*,
                              const double*, double, int, int);
}  // namespace rx

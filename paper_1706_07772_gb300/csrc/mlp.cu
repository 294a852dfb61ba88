// (e5) Learned QEq warm start: per-atom environment descriptors, a per-element MLP
// (192 -> 64 -> 64 -> 1, SiLU) predicting the atom's charge, and its training.
//
// Paper: Sec. 3.3 starts the QEq CG from an extrapolated guess; here a network trained on
// charges the method itself produced supplies another guess. The CG still runs to the
// same tolerance, so the guess moves only its starting point (the charges do not change
// beyond the tolerance).
//
// Descriptors (192 per atom), for each neighbour element e:
//   radial  G_R[e,k] = sum_{j of e, r < 6 A} exp(-eta_r (r - mu_k)^2) fc(r), k = 0..31,
//           mu_k = 0.8 + k 5.2/31, eta_r = 1 / (2 (5.2/31)^2), fc(r) = (cos(pi r/rc) + 1)/2
//   angular G_A[e,(z,a,l)] = 2^(1-zeta) sum over ordered pairs (j,k), j != k, r < 3.5 A,
//           j of e: (1 + lambda cos theta_jik)^zeta exp(-eta (r_ij^2 + r_ik^2)) fc fc,
//           zeta in {1,2,4,8}, eta in {0.05, 0.3}, lambda in {+1,-1}, index 4z + 2a + l
// laid out per element as [32 radial, 16 angular]. Network per centre element t:
//   z1 = x~ W1 + b1, a1 = silu(z1), z2 = a1 W2 + b2, a2 = silu(z2), y = a2 . w3 + b3,
// x~ = (x - mean) inv_std. Parameter vector per element: W1[192][64], b1[64], W2[64][64],
// b2[64], w3[64], b3 (16,577 floats).
//
// Inference runs on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// TMEM) over tiles of 128 atoms of one element; training runs FP32 forward / backward /
// Adam kernels (small contractions, deterministic fixed-order reductions).
#include <cuda_bf16.h>

#include "reax_internal.cuh"

namespace {

constexpr int NT = rx::MLP_NT, NR = 32, NA = 16, NE = NR + NA, NF = NT * NE, HID = rx::MLP_HID;
constexpr int NPAR = rx::MLP_NPAR;
static_assert(NF == rx::MLP_NF, "descriptor layout");
constexpr int O_W1 = 0, O_B1 = NF * HID, O_W2 = O_B1 + HID, O_B2 = O_W2 + HID * HID, O_W3 = O_B2 + HID,
              O_B3 = O_W3 + HID;
static_assert(O_B3 + 1 == NPAR, "parameter layout");
constexpr float RC_R = 6.0f, RC_A = 3.5f, MU0 = 0.8f, DMU = 5.2f / 31.0f;
constexpr int DESC_NB = 192;    // neighbours within 6 A kept per atom (more: error flag)
constexpr int DESC_NBA = 64;    // neighbours within 3.5 A

__device__ __forceinline__ float cutoff(float r, float rc) {
  return r < rc ? 0.5f * (__cosf(3.14159265358979f * r / rc) + 1.0f) : 0.0f;
}

// descriptors: warp per atom. The neighbours within 6 A (near rows: r < r_bond = 5 A;
// far rows filtered) are compacted into shared memory; lane k then sums radial feature k
// for the four elements, and the angular features are summed per element over the
// ordered pairs of the 3.5 A neighbours (lanes over pairs, fixed-order warp reduction).
constexpr int DW = 4;           // warps per block
// gate (or null): the QEq history state {newest s, newest t, usable solutions}; with a
// usable history the extrapolated start is kept, so the learned guess is not computed
__device__ __forceinline__ bool gated_off(const int* gate) { return gate && gate[2] > 0; }

__global__ void __launch_bounds__(DW * 32) k_desc(Sys s, FarList f, float* D, int n, const int* gate) {
  __shared__ float sr[DW][DESC_NB], sx[DW][DESC_NB], sy[DW][DESC_NB], sz[DW][DESC_NB];
  __shared__ int st[DW][DESC_NB];
  if (gated_off(gate)) return;                         // grid-uniform
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * DW + w;
  if (i >= n) return;                                  // warp-uniform
  const int r = s.rep[i];
  int m = 0;
  for (int part = 0; part < 2; ++part) {
    const int cnt = part == 0 ? f.cntn[i] : f.cnt[i];
    const int* jj = part == 0 ? f.jn + (size_t)i * f.capn : f.j + (size_t)i * f.cap;
    const uint8_t* cc = part == 0 ? f.sn + (size_t)i * f.capn : f.s + (size_t)i * f.cap;
    for (int b = 0; b < cnt; b += 32) {
      const int k = b + lane;
      float dx = 0, dy = 0, dz = 0, rr = 1e30f;
      int tj = 0;
      if (k < cnt) {
        float4 hj, lj;
        PairVec<float>::getv(s, i, jj[k], cc[k], r, dx, dy, dz, hj, lj);
        rr = sqrtf(dx * dx + dy * dy + dz * dz);
        tj = rec_type(lj.w);
      }
      const bool in = rr < RC_R;
      const unsigned mk = __ballot_sync(0xffffffffu, in);
      const int pos = m + __popc(mk & ((1u << lane) - 1u));
      if (in && pos < DESC_NB) {
        sr[w][pos] = rr; sx[w][pos] = dx; sy[w][pos] = dy; sz[w][pos] = dz; st[w][pos] = tj;
      }
      m += __popc(mk);
    }
  }
  if (m > DESC_NB) {
    if (lane == 0) atomicOr(s.err, ERR_CAP_DESC);
    m = DESC_NB;
  }
  __syncwarp();
  float* out = D + (size_t)i * NF;
  // radial: lane = k
  {
    const float mu = MU0 + lane * DMU, eta = 1.0f / (2.0f * DMU * DMU);
    float acc[NT] = {0, 0, 0, 0};
    for (int p = 0; p < m; ++p) {
      const float rr = sr[w][p];
      const float g = expf(-eta * (rr - mu) * (rr - mu)) * cutoff(rr, RC_R);
      const int t = st[w][p];
#pragma unroll
      for (int e = 0; e < NT; ++e) acc[e] += t == e ? g : 0.0f;
    }
#pragma unroll
    for (int e = 0; e < NT; ++e) out[e * NE + lane] = acc[e];
  }
  // angular: compact the 3.5 A neighbours to the front (in order), then pairs per element
  int ma = 0;
  for (int b = 0; b < m; b += 32) {
    const int p = b + lane;
    const bool in = p < m && sr[w][p] < RC_A;
    float rr = 0, dx = 0, dy = 0, dz = 0;
    int tj = 0;
    if (in) { rr = sr[w][p]; dx = sx[w][p]; dy = sy[w][p]; dz = sz[w][p]; tj = st[w][p]; }
    const unsigned mk = __ballot_sync(0xffffffffu, in);
    const int pos = ma + __popc(mk & ((1u << lane) - 1u));
    __syncwarp();                                      // reads of this chunk before writes
    if (in && pos < DESC_NBA) { sr[w][pos] = rr; sx[w][pos] = dx; sy[w][pos] = dy; sz[w][pos] = dz; st[w][pos] = tj; }
    __syncwarp();
    ma += __popc(mk);
  }
  if (ma > DESC_NBA) {
    if (lane == 0) atomicOr(s.err, ERR_CAP_DESC);
    ma = DESC_NBA;
  }
  for (int e = 0; e < NT; ++e) {
    float acc[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) acc[q] = 0.0f;
    for (int t = lane; t < ma * ma; t += 32) {
      const int p = t / ma, q = t % ma;
      if (p == q || st[w][p] != e) continue;
      const float rp = sr[w][p], rq = sr[w][q];
      const float c = (sx[w][p] * sx[w][q] + sy[w][p] * sy[w][q] + sz[w][p] * sz[w][q]) / (rp * rq);
      const float ff = cutoff(rp, RC_A) * cutoff(rq, RC_A);
      const float s2 = rp * rp + rq * rq;
      const float ra0 = expf(-0.05f * s2) * ff, ra1 = expf(-0.3f * s2) * ff;
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        const float b1 = 1.0f + (l == 0 ? c : -c);
        const float b2 = b1 * b1, b4 = b2 * b2, b8 = b4 * b4;
        const float pw[4] = {b1, 0.5f * b2, 0.125f * b4, 0.0078125f * b8};   // 2^(1-zeta) (1 + l c)^zeta
#pragma unroll
        for (int z = 0; z < 4; ++z) {
          acc[4 * z + 0 + l] += pw[z] * ra0;
          acc[4 * z + 2 + l] += pw[z] * ra1;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NA; ++q) acc[q] = warp_sumf(acc[q]);
    float v = 0.0f;
#pragma unroll
    for (int q = 0; q < NA; ++q) v = lane == q ? acc[q] : v;
    if (lane < NA) out[e * NE + NR + lane] = v;
  }
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_g(float z) {
  const float sg = 1.0f / (1.0f + __expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}

// FP32 forward for training: thread per sample; stores z1, z2 and y
__global__ void k_fwd32(const float* X, const int* type, int m, const float* theta, const float* mean,
                        const float* inv, float* Z1, float* Z2, float* Y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  const float* th = theta + (size_t)type[b] * NPAR;
  float z[HID];
#pragma unroll
  for (int j = 0; j < HID; ++j) z[j] = th[O_B1 + j];
  const float* x = X + (size_t)b * NF;
  for (int k = 0; k < NF; ++k) {
    const float xk = (x[k] - mean[k]) * inv[k];
    const float* wr = th + O_W1 + k * HID;
#pragma unroll
    for (int j = 0; j < HID; ++j) z[j] = fmaf(xk, wr[j], z[j]);
  }
  float* z1 = Z1 + (size_t)b * HID;
#pragma unroll
  for (int j = 0; j < HID; ++j) z1[j] = z[j];
  float u[HID];
#pragma unroll
  for (int j = 0; j < HID; ++j) u[j] = th[O_B2 + j];
  for (int k = 0; k < HID; ++k) {
    const float ak = silu_f(z1[k]);
    const float* wr = th + O_W2 + k * HID;
#pragma unroll
    for (int j = 0; j < HID; ++j) u[j] = fmaf(ak, wr[j], u[j]);
  }
  float* z2 = Z2 + (size_t)b * HID;
  float y = th[O_B3];
#pragma unroll
  for (int j = 0; j < HID; ++j) {
    z2[j] = u[j];
    y = fmaf(silu_f(u[j]), th[O_W3 + j], y);
  }
  Y[b] = y;
}

// FP32 backward per sample: dL/dy = 2 (y - q) / m; writes dz1 and dz2 (per-sample
// gradients of the pre-activations); the loss contribution goes to L[b]
__global__ void k_bwd32(const int* type, int m, const float* theta, const float* Q, const float* Z1,
                        const float* Z2, const float* Y, float* DZ1, float* DZ2, float* L) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  const float* th = theta + (size_t)type[b] * NPAR;
  const float e = Y[b] - Q[b];
  L[b] = e * e;
  const float dy = 2.0f * e / (float)m;
  const float* z2 = Z2 + (size_t)b * HID;
  float* dz2 = DZ2 + (size_t)b * HID;
  float g2[HID];
#pragma unroll
  for (int j = 0; j < HID; ++j) {
    g2[j] = dy * th[O_W3 + j] * silu_g(z2[j]);
    dz2[j] = g2[j];
  }
  const float* z1 = Z1 + (size_t)b * HID;
  float* dz1 = DZ1 + (size_t)b * HID;
  for (int k = 0; k < HID; ++k) {
    const float* wr = th + O_W2 + k * HID;
    float a = 0.0f;
#pragma unroll
    for (int j = 0; j < HID; ++j) a = fmaf(wr[j], g2[j], a);
    dz1[k] = a * silu_g(z1[k]);
  }
}

// weight gradients, one thread per parameter of one element and chunk of WG_CHUNK of that
// element's samples (idx[off[t] .. off[t+1]), in index order): partial sums part[c][gid],
// then summed over the chunks in order by k_wgrad_sum (deterministic)
constexpr int WG_CHUNK = rx::MLP_WG_CHUNK;
__global__ void k_wgrad(const float* X, const int* idx, const int* off, const float* theta, const float* mean,
                        const float* inv, const float* Z1, const float* Z2, const float* DZ1, const float* DZ2,
                        const float* Y, const float* Q, int m, float* part) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= NT * NPAR) return;
  const int t = gid / NPAR, p = gid % NPAR;
  float acc = 0.0f;
  const int a = min(off[t] + (int)blockIdx.y * WG_CHUNK, off[t + 1]);
  const int bnd = min(a + WG_CHUNK, off[t + 1]);
  if (p < O_B1) {                                      // W1[k][j] = sum x~_k dz1_j
    const int k = p / HID, j = p % HID;
    for (int s = a; s < bnd; ++s) {
      const int b = idx[s];
      acc = fmaf((X[(size_t)b * NF + k] - mean[k]) * inv[k], DZ1[(size_t)b * HID + j], acc);
    }
  } else if (p < O_W2) {                               // b1[j]
    const int j = p - O_B1;
    for (int s = a; s < bnd; ++s) acc += DZ1[(size_t)idx[s] * HID + j];
  } else if (p < O_B2) {                               // W2[k][j] = sum a1_k dz2_j
    const int k = (p - O_W2) / HID, j = (p - O_W2) % HID;
    for (int s = a; s < bnd; ++s) {
      const int b = idx[s];
      acc = fmaf(silu_f(Z1[(size_t)b * HID + k]), DZ2[(size_t)b * HID + j], acc);
    }
  } else if (p < O_W3) {                               // b2[j]
    const int j = p - O_B2;
    for (int s = a; s < bnd; ++s) acc += DZ2[(size_t)idx[s] * HID + j];
  } else if (p < O_B3) {                               // w3[j] = sum a2_j dy
    const int j = p - O_W3;
    for (int s = a; s < bnd; ++s) {
      const int b = idx[s];
      acc = fmaf(silu_f(Z2[(size_t)b * HID + j]), 2.0f * (Y[b] - Q[b]) / (float)m, acc);
    }
  } else {                                             // b3
    for (int s = a; s < bnd; ++s) acc += 2.0f * (Y[idx[s]] - Q[idx[s]]) / (float)m;
  }
  part[(size_t)blockIdx.y * (NT * NPAR) + gid] = acc;
}
__global__ void k_wgrad_sum(const float* part, int nchunk, float* G) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= NT * NPAR) return;
  float s = 0.0f;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * (NT * NPAR) + gid];
  G[gid] = s;
}

__global__ void k_adam(float* theta, const float* g, float* mo, float* vo, int np, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const float m = b1 * mo[k] + (1.0f - b1) * g[k];
  const float v = b2 * vo[k] + (1.0f - b2) * g[k] * g[k];
  mo[k] = m;
  vo[k] = v;
  theta[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// per-feature mean and 1/std over rows of X (thread per feature, rows in order, FP64 sums)
__global__ void k_stats(const float* X, int64_t rows, float* mean, float* inv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NF) return;
  double s = 0.0, s2 = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    const double v = X[r * NF + k];
    s += v;
    s2 += v * v;
  }
  const double mu = s / (double)rows;
  const double var = s2 / (double)rows - mu * mu;
  mean[k] = (float)mu;
  inv[k] = var > 1e-24 ? (float)(1.0 / sqrt(var)) : 0.0f;
}

__global__ void k_sumsq(const float* L, int m, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int b = threadIdx.x; b < m; b += blockDim.x) v += L[b];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t / (double)m;
  }
}


// ------------------------------------------------------------------ tensor-core inference
// One CTA (4 warps) per tile of 128 atoms of one element, persistent over tiles. Operands
// live in shared memory in the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices (8 x 8 BF16), the K-adjacent core matrices 128 B apart (leading byte
// offset) and the 8-row groups (K/8) x 128 B apart (stride byte offset). Thread 0 issues
// tcgen05.mma (kind::f16: BF16 A and B, FP32 accumulator in TMEM, M = 128, N = 64, K = 16
// per instruction) and commits to an mbarrier; warp w reads TMEM lanes 32w..32w+31 (its
// rows) with tcgen05.ld. Layer 1: A = x~ (128 x 192), B = W1^T (64 x 192); the SiLU output
// goes back to shared memory as the layer-2 A operand (128 x 64) against B = W2^T; the
// last layer (64 -> 1) is a dot product in registers.
constexpr int TM = 128;
constexpr uint32_t TC_SMEM = 200 * 1024;   // 96 KB of operands, the rest keeps every
                                           // descriptor reading inside the allocation
constexpr uint32_t SM_A1 = 0, SM_B1 = 49152, SM_A2 = 73728, SM_B2 = 90112;
constexpr uint32_t IDESC = (1u << 4)                       // D: FP32
                           | (1u << 7) | (1u << 10)        // A, B: BF16
                           | ((uint32_t)(HID >> 3) << 17)  // N = 64
                           | ((uint32_t)(TM >> 4) << 24);  // M = 128
constexpr long long TC_SPIN_LIMIT = 4000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// byte offset of element (row, k) of a K-major core-matrix operand with K columns
__device__ __forceinline__ uint32_t cm_off(int row, int k, int K) {
  return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}
// shared-memory matrix descriptor: start address, leading / stride byte offsets (>> 4),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(a), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (long long k = 0; k < TC_SPIN_LIMIT; ++k)
    if (mbar_try(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
               "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *(const uint32_t*)&h;
}

// Xp: packed normalised inputs [rows][192] BF16 (row p is atom perm[p]); tiles t cover rows
// [rows_off[t], rows_off[t+1]) (<= 128) of element tile_type[t]; W1t[t][j][k] = W1[k][j],
// W2t[t][j][k] = W2[k][j] (BF16); fp[t] = {b1[64], b2[64], w3[64], b3} (FP32)
__global__ void __launch_bounds__(128, 1) k_mlp_tc(const __nv_bfloat16* __restrict__ Xp, const int* tile_type,
                                                   const int* rows_off, const int* perm, int ntile,
                                                   const __nv_bfloat16* __restrict__ W1t,
                                                   const __nv_bfloat16* __restrict__ W2t, const float* fp,
                                                   float* y_out, int* err, const int* gate) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  if (gated_off(gate)) return;                         // grid-uniform, before any TMEM allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" :: "r"(smem_u32(&tmem_slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(smem_u32(&mbar));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t sA1 = smem_u32(smem + SM_A1), sB1 = smem_u32(smem + SM_B1);
  const uint32_t sA2 = smem_u32(smem + SM_A2), sB2 = smem_u32(smem + SM_B2);
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's TMEM lanes
  uint32_t parity = 0;
  bool ok = true;
  for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
    const int ty = tile_type[t], r0 = rows_off[t], nr = rows_off[t + 1] - r0;
    for (int e = tid; e < TM * (NF / 8); e += 128) {            // A1: 16-byte chunks of x~
      const int row = e / (NF / 8), kc = e % (NF / 8);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < nr) v = *(const uint4*)(Xp + (size_t)(r0 + row) * NF + kc * 8);
      *(uint4*)(smem + SM_A1 + cm_off(row, kc * 8, NF)) = v;
    }
    for (int e = tid; e < HID * (NF / 8); e += 128) {           // B1 = W1^T
      const int row = e / (NF / 8), kc = e % (NF / 8);
      *(uint4*)(smem + SM_B1 + cm_off(row, kc * 8, NF)) =
          *(const uint4*)(W1t + ((size_t)ty * HID + row) * NF + kc * 8);
    }
    for (int e = tid; e < HID * (HID / 8); e += 128) {          // B2 = W2^T
      const int row = e / (HID / 8), kc = e % (HID / 8);
      *(uint4*)(smem + SM_B2 + cm_off(row, kc * 8, HID)) =
          *(const uint4*)(W2t + ((size_t)ty * HID + row) * HID + kc * 8);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      for (int k = 0; k < NF / 16; ++k)
        tc_mma(tmem, smem_desc(sA1 + 256 * k, 128, (NF / 8) * 128), smem_desc(sB1 + 256 * k, 128, (NF / 8) * 128), k > 0);
      tc_commit(mb);
    }
    ok = mbar_wait(mb, parity);
    parity ^= 1;
    tc_fence_after();
    const float* f = fp + (size_t)ty * (3 * HID + 1);
    const int row = 32 * warp + lane;
    float h[HID];
    if (ok) {
#pragma unroll
      for (int c = 0; c < HID; c += 16) tmem_ld16(trow + c, h + c);
      tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < HID; c += 8) {                         // a1 = silu(z1) -> A2
        uint4 v;
        v.x = pack_bf16(silu_f(h[c + 0] + f[c + 0]), silu_f(h[c + 1] + f[c + 1]));
        v.y = pack_bf16(silu_f(h[c + 2] + f[c + 2]), silu_f(h[c + 3] + f[c + 3]));
        v.z = pack_bf16(silu_f(h[c + 4] + f[c + 4]), silu_f(h[c + 5] + f[c + 5]));
        v.w = pack_bf16(silu_f(h[c + 6] + f[c + 6]), silu_f(h[c + 7] + f[c + 7]));
        *(uint4*)(smem + SM_A2 + cm_off(row, c, HID)) = v;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ok && tid == 0) {
      for (int k = 0; k < HID / 16; ++k)
        tc_mma(tmem, smem_desc(sA2 + 256 * k, 128, (HID / 8) * 128), smem_desc(sB2 + 256 * k, 128, (HID / 8) * 128), k > 0);
      tc_commit(mb);
    }
    if (ok) {
      ok = mbar_wait(mb, parity);
      parity ^= 1;
    }
    tc_fence_after();
    if (ok) {
#pragma unroll
      for (int c = 0; c < HID; c += 16) tmem_ld16(trow + c, h + c);
      tmem_wait_ld();
      float y = f[3 * HID];
#pragma unroll
      for (int c = 0; c < HID; ++c) y = fmaf(silu_f(h[c] + f[HID + c]), f[2 * HID + c], y);
      if (row < nr) y_out[perm[r0 + row]] = y;
    }
    tc_fence_before();
    __syncthreads();                                             // TMEM and smem reused next
    tc_fence_after();
  }
  if (!ok) {                                                     // let the last MMAs land
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    mbar_wait(mb, parity);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" :: "r"(tmem) : "memory");
}

// x~ = (x - mean) inv_std in BF16, packed in tile order: row p <- atom perm[p]
__global__ void k_mlp_pack(const float* D, const int* perm, int rows, const float* mean, const float* inv,
                           __nv_bfloat16* Xp, const int* gate) {
  if (gated_off(gate)) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * NF) return;
  const int p = (int)(e / NF), k = (int)(e % NF);
  Xp[e] = __float2bfloat16_rn((D[(size_t)perm[p] * NF + k] - mean[k]) * inv[k]);
}

// BF16 transposed weights and FP32 bias/output-layer vectors from the FP32 parameters
__global__ void k_mlp_weights(const float* theta, __nv_bfloat16* W1t, __nv_bfloat16* W2t, float* fp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = HID * NF + HID * HID + 3 * HID + 1;
  if (e >= NT * per) return;
  const int t = e / per, q = e % per;
  const float* th = theta + (size_t)t * NPAR;
  if (q < HID * NF) {
    const int j = q / NF, k = q % NF;
    W1t[(size_t)t * HID * NF + q] = __float2bfloat16_rn(th[O_W1 + k * HID + j]);
  } else if (q < HID * NF + HID * HID) {
    const int q2 = q - HID * NF, j = q2 / HID, k = q2 % HID;
    W2t[(size_t)t * HID * HID + q2] = __float2bfloat16_rn(th[O_W2 + k * HID + j]);
  } else {
    const int q3 = q - HID * NF - HID * HID;                     // b1, b2, w3, b3
    fp[(size_t)t * (3 * HID + 1) + q3] =
        q3 < HID ? th[O_B1 + q3] : q3 < 2 * HID ? th[O_B2 + q3 - HID] : q3 < 3 * HID ? th[O_W3 + q3 - 2 * HID] : th[O_B3];
  }
}

}  // namespace

namespace rx {

void mlp_weights(const Launch& L, const float* theta, MlpInfer& w) {
  k_mlp_weights<<<(NT * (HID * NF + HID * HID + 3 * HID + 1) + 255) / 256, 256, 0, L.st>>>(theta, (__nv_bfloat16*)w.W1t, (__nv_bfloat16*)w.W2t, w.fp);
  *L.count += 1;
}

void mlp_infer(const Launch& L, const float* D, const MlpTiles& T, const float* mean, const float* inv,
               MlpInfer& w, float* y_out, int* err, int nsm, const int* gate) {
  const int64_t tot = (int64_t)T.rows * NF;
  k_mlp_pack<<<(unsigned)((tot + 255) / 256), 256, 0, L.st>>>(D, T.perm, T.rows, mean, inv, (__nv_bfloat16*)w.Xp,
                                                               gate);
  const int grid = T.ntile < nsm ? T.ntile : nsm;
  if (grid > 0)
    k_mlp_tc<<<grid, 128, TC_SMEM, L.st>>>((const __nv_bfloat16*)w.Xp, T.tile_type, T.rows_off, T.perm, T.ntile, (const __nv_bfloat16*)w.W1t, (const __nv_bfloat16*)w.W2t, w.fp, y_out, err, gate);
  *L.count += 2;
}

int mlp_tc_setup() {
  return (int)cudaFuncSetAttribute((const void*)k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

void mlp_descriptors(const Launch& L, Sys s, FarList f, float* D, const int* gate) {
  k_desc<<<(s.n + DW - 1) / DW, DW * 32, 0, L.st>>>(s, f, D, s.n, gate);
  *L.count += 1;
}

void mlp_stats(const Launch& L, const float* X, int64_t rows, float* mean, float* inv) {
  k_stats<<<(NF + 63) / 64, 64, 0, L.st>>>(X, rows, mean, inv);
  *L.count += 1;
}

void mlp_loss_grad(const Launch& L, const float* X, const int* type, const int* idx, const int* off, const float* Q,
                   int m, const float* theta, const float* mean, const float* inv, MlpScratch& w, float* G,
                   double* loss) {
  k_fwd32<<<(m + 127) / 128, 128, 0, L.st>>>(X, type, m, theta, mean, inv, w.z1, w.z2, w.y);
  k_bwd32<<<(m + 127) / 128, 128, 0, L.st>>>(type, m, theta, Q, w.z1, w.z2, w.y, w.dz1, w.dz2, w.l);
  const int nchunk = (m + WG_CHUNK - 1) / WG_CHUNK;     // enough for any one element
  k_wgrad<<<dim3((NT * NPAR + 127) / 128, nchunk), 128, 0, L.st>>>(X, idx, off, theta, mean, inv, w.z1, w.z2, w.dz1,
                                                                  w.dz2, w.y, Q, m, w.part);
  k_wgrad_sum<<<(NT * NPAR + 255) / 256, 256, 0, L.st>>>(w.part, nchunk, G);
  k_sumsq<<<1, 256, 0, L.st>>>(w.l, m, loss);
  *L.count += 5;
}

void mlp_forward32(const Launch& L, const float* X, const int* type, int m, const float* theta, const float* mean,
                   const float* inv, MlpScratch& w) {
  k_fwd32<<<(m + 127) / 128, 128, 0, L.st>>>(X, type, m, theta, mean, inv, w.z1, w.z2, w.y);
  *L.count += 1;
}

void mlp_adam(const Launch& L, float* theta, const float* g, float* mo, float* vo, int step, float lr) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(NT * NPAR + 255) / 256, 256, 0, L.st>>>(theta, g, mo, vo, NT * NPAR, lr, b1, b2, 1e-8f, c1, c2);
  *L.count += 1;
}

}  // namespace rx

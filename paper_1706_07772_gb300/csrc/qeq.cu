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
// (w = H p is carried as H z + beta w, so H is read once per iteration.) Each phase writes
// per-chunk partial dot products and ends in a grid barrier; after it every block reduces
// all partials itself, in one fixed order, so every block holds bit-identical alpha, beta
// and convergence flags without a second synchronisation (the partials are double-
// buffered: a block that runs ahead writes the other buffer). Convergence per system and
// replica: ||r||_2 <= tol ||b||_2; a converged system freezes while the other continues.
// Barrier waits are bounded.
//
// GB300 runs FP64 at 1/64 of the FP32 rate: about two FP64 operations per clock per SM,
// so one FP64 warp instruction holds the SM's FP64 pipe for ~16 cycles whatever its active
// lanes. The kernel therefore keeps FP64 to the per-row vector updates, packed densely
// (thread t <-> row t of the block, so ~rows/32 warps issue them), and to a few
// multi-value warp reductions; the SpMV itself runs in the path precision with its row
// sums left in shared memory until the dense update reads them.
#include "reax_internal.cuh"

namespace {

constexpr int NQ = 8;          // partial-sum slots per chunk
constexpr int NS = 16;         // scalars per replica
// scalar slots per replica
enum { S_RHO_S = 0, S_RHO_T, S_AL_S, S_AL_T, S_BE_S, S_BE_T, S_BB_S, S_BB_T, S_ACT_S, S_ACT_T, S_MU, S_USE };
// row state of a block (doubles per row; U holds the SpMV row sums as two values of the
// path type)
enum { V_XS = 0, V_XT, V_RS, V_RT, V_PS, V_PT, V_WS, V_WT, V_ZS, V_ZT, V_ETA, V_IETA, V_U, V_U2, NV_STATE };
static_assert(NV_STATE == rx::QEQ_NV_STATE, "row state layout");
static_assert(NS + NQ == rx::QEQ_SCAL_PER_REP, "scalar layout");
constexpr int MAXC = 32;       // chunk bounds cached in shared memory per block

template <typename R>
struct CG {
  int n, nrep, nchunk, max_iter;
  double tol2;
  const int* type;
  const int* cnt;                          // far part of each row (r_bond <= r < r_nb)
  const int* col;
  const R* H;
  int cap;
  const int* cntn;                         // near part of each row
  const int* coln;
  const R* Hn;
  int capn;
  const double *eta, *chi, *ieta;          // per type (double); ieta = 1/eta
  const float* binv;                       // block-Jacobi inverses (null: Jacobi, z = r / eta)
  // solution history rings (rx::QEQ_HIST slots each) and their device state hst = {slot of the
  // newest s, slot of the newest t, usable entries}; read by every block at the start,
  // advanced by block 0 at the end (the new solutions go to the oldest slots)
  double *hist_s, *hist_t;
  int* hst;
  int warm;                                // 1: extrapolate from the history, 0: start at 0
  const double* wext;                      // [QEQ_NPRED][2][H+1][H] guess weights (H = QEQ_HIST)
  int* pred;                               // [2*nrep] predictor in use per replica and system
  int adapt;                               // 1: re-pick the predictor after every solve
  const float* qhat;                       // learned charges (or null): a second guess for s
  int* mlp_used;                           // [nrep] 1 where the learned guess was kept
  void* zg;                                // interleaved (s, t) SpMV operand: float2 or double2
  double* q;
  float* qf;
  float4* ph;                              // packed records: charge field (may be null)
  double* part;                            // [2][NQ][nchunk] chunk partials, two buffers
  double* scal;                            // [grid][nrep*(NS+NQ)+4] scalars, unless in shared memory
  double* state;                           // [grid][NV_STATE][rows_blk] row state, unless in shared memory
  int rows_blk;                            // most rows any block owns
  int scal_smem, state_smem;               // 1: kept in dynamic shared memory
  int ring_bytes;                          // SpMV ring at the start of dynamic shared memory
  int bj_smem;                             // 1: block inverses staged in shared memory after the state
  const int* chunk_lo;                     // [nchunk+1] rows
  const int* chunk_rep;                    // [nchunk]
  const int* rep_chunk;                    // [nrep+1] chunk ranges per replica
  int* iters;                              // [2*nrep]
  unsigned long long* spmv_total;          // SpMVs performed by all solves (diagnostic)
  GridBar* bar;
  long long bar_limit;                     // SM cycles a grid-barrier wait may take
  int* err;
};

// Bounded grid barrier (all blocks co-resident: cooperative launch). The arrival counter
// is zeroed before the launch and only grows: the k-th barrier completes when it reaches
// k * gridDim.x (`target` counts this block's barriers). Thread 0 adds with acquire-release
// semantics (publishes the block's writes, ordered before it by __syncthreads, and takes
// those of the blocks that arrived earlier) and polls with acquire loads; no reset, so a
// barrier costs one atomic round trip plus the wait for the last block. The wait gives up
// after `limit` SM cycles (BAR_CYCLE_LIMIT unless the context set another) and raises
// ERR_TIMEOUT; every block then leaves the kernel at its next barrier (no cp.async copy is
// in flight at a barrier: the SpMV ring drains before it returns).
__device__ bool grid_barrier(GridBar* bar, int* err, unsigned& target, long long limit) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    unsigned cur;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(cur) : "l"(&bar->arrive) : "memory");
    cur += 1u;
    const long long t0 = clock64();
    while ((int)(cur - target) < 0) {
      if (clock64() - t0 > limit) {
        atomicOr(err, ERR_TIMEOUT);
        break;
      }
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->arrive) : "memory");
    }
  }
  __syncthreads();
  return !(*((volatile int*)err) & ERR_TIMEOUT);
}

// Sum NVP values (a power of two) over the 32 lanes with NVP - 1 + 5 - log2(NVP) FP64 adds
// per lane instead of 5 NVP: each exchange step halves the values a lane keeps (the lower
// lane of a pair keeps the first half, the upper the second), then plain butterflies
// finish. Returns the total of slot `slot`, the same on all 32/NVP lanes of a group (IEEE
// addition commutes, so partners agree bit for bit). Fixed order: deterministic.
template <int NVP>
__device__ __forceinline__ double warp_reduce_multi(double* v, int& slot) {
  const int lane = threadIdx.x & 31;
  slot = 0;
  int s = 16;
#pragma unroll
  for (int c = NVP; c > 1; c >>= 1, s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < c / 2; ++k) {
      const double send = up ? v[k] : v[k + c / 2];
      const double keep = up ? v[k + c / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
    slot = 2 * slot + (up ? 1 : 0);
  }
  double t = v[0];
#pragma unroll
  for (; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
  return t;
}
template <int NV> struct Pow2 { static constexpr int v = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : 8; };

// per-replica totals of the first NV slots of partial buffer pb -> red[r*NQ + q]: one warp
// per replica, lane l sums chunks l, l+32, ... in order, then one multi-value butterfly
// (every block computes bit-identical totals)
template <int NV, typename R>
__device__ __forceinline__ void reduce_parts(const CG<R>& a, int pb, double* red) {
  constexpr int NVP = Pow2<NV>::v;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* P = a.part + (size_t)pb * NQ * a.nchunk;
  constexpr int U = NV <= 2 ? 4 : (NV <= 4 ? 2 : 1);      // chunks per lane in flight
  for (int r = wid; r < a.nrep; r += nw) {
    double v[NVP];
#pragma unroll
    for (int q = 0; q < NVP; ++q) v[q] = 0.0;
    const int c1 = a.rep_chunk[r + 1];
    int c = a.rep_chunk[r] + lane;
    for (; c + 32 * (U - 1) < c1; c += 32 * U) {
      double t[U][NV];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < NV; ++q) t[u][q] = __ldcg(P + (size_t)q * a.nchunk + c + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] += t[u][q];
    }
    for (; c < c1; c += 32)
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] += __ldcg(P + (size_t)q * a.nchunk + c);
    int slot;
    const double t = warp_reduce_multi<NVP>(v, slot);
    if ((lane & (32 / NVP - 1)) == 0 && slot < NV) red[r * NQ + slot] = t;
  }
  __syncthreads();
}

// chunk partial sums of NV per-thread values -> part[pb][q][chunk]. Threads hold values
// only for rows t < nr (dense map), so warps past the last row contribute zeros without
// arithmetic; warp totals are combined by warp 0 in warp order (deterministic).
template <int NV, typename R>
__device__ __forceinline__ void block_sum(const CG<R>& a, double* v, int nr, int pb, int chunk) {
  constexpr int NVP = Pow2<NV>::v;
  __shared__ double sh[32][NVP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double w[NVP];
#pragma unroll
  for (int q = 0; q < NVP; ++q) w[q] = q < NV ? v[q] : 0.0;
  if (wid * 32 < nr) {
    int slot;
    const double t = warp_reduce_multi<NVP>(w, slot);
    if ((lane & (32 / NVP - 1)) == 0) sh[wid][slot] = t;
  } else if (lane < NVP) {
    sh[wid][lane] = 0.0;
  }
  __syncthreads();
  if (wid == 0) {
    double u[NVP];
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NVP; ++q) u[q] = lane < nw ? sh[lane][q] : 0.0;
    int slot;
    const double t = warp_reduce_multi<NVP>(u, slot);
    if ((lane & (32 / NVP - 1)) == 0 && slot < NV) a.part[((size_t)pb * NQ + slot) * a.nchunk + chunk] = t;
  }
  __syncthreads();
}

// (H v)_i for the two systems, warp per row, both right-hand sides gathered in one load of
// the interleaved copy zg[j] = (v_s[j], v_t[j]). Lane l takes entries l, l+32, l+64, l+96 of
// each 128-entry group: the column and H loads of a group are coalesced, and the gathers of
// one load instruction fall on 32 consecutive list entries (a few neighbouring cells, so a
// few cache lines). The next group's column/H loads are issued before this group's
// multiply-adds. Padding lanes gather zg[i] with h = 0 (adds an exact zero).
// FP64 path: FP64 products and sums. Mixed path: H and zg in FP32, FP32 products and
// per-lane partial sums (about 13 terms per lane), lanes combined by an FP32 butterfly.
template <typename R> struct G2;
template <> struct G2<float> { using T = float2; };
template <> struct G2<double> { using T = double2; };

__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float warp_total(float v) { return warp_sumf(v); }
__device__ __forceinline__ double warp_total(double v) { return warp_sum(v); }

// streamed matrix loads: read-only for the kernel's lifetime, kept out of L1 (the L1 holds
// the gathered vector)
__device__ __forceinline__ int ld_stream(const int* p) {
  int v;
  asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

template <typename R>
__device__ __forceinline__ void spmv_part(const int* cnt, const int* col, const R* H, int cap, int i,
                                          const typename G2<R>::T* zg, R& sf, R& tf) {
  using T = typename G2<R>::T;
  const int lane = threadIdx.x & 31;
  const int* cr = col + (size_t)i * cap;
  const R* hr = H + (size_t)i * cap;
  const int nf = ld_stream(cnt + i);
  int j[4];
  R h[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = lane + 32 * u;
    j[u] = i;
    h[u] = R(0);
    if (k < nf) {
      j[u] = ld_stream(cr + k);
      h[u] = ld_stream(hr + k);
    }
  }
  for (int k0 = 0; k0 < nf; k0 += 128) {
    T z[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) z[u] = zg[j[u]];
    int jn[4];
    R hn[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 128 + lane + 32 * u;
      jn[u] = i;
      hn[u] = R(0);
      if (k < nf) {
        jn[u] = ld_stream(cr + k);
        hn[u] = ld_stream(hr + k);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sf = fmaR(h[u], z[u].x, sf);
      tf = fmaR(h[u], z[u].y, tf);
      j[u] = jn[u];
      h[u] = hn[u];
    }
  }
}

// Mixed path SpMV of a warp's run of rows, with the matrix streamed through shared memory.
// The work is a sequence of items: up to 128 consecutive entries of one part (near, then
// far) of one row. Each warp owns SP_SLOTS ring slots of one item (128 columns, 128 H
// values); lane l fills bytes 16l..16l+15 of both halves with cp.async (16-byte copies
// that bypass L1 and hold no registers while in flight), zero-filling past the part's
// count. The warp keeps SP_SLOTS - 1 items in flight ahead of the one it multiplies, across
// row boundaries, so the stream does not wait on the gathers. Consuming an item, lane l
// reads entries l, l+32, l+64, l+96 (the gathers of one load instruction fall on 32
// consecutive list entries, a few cache lines) and refills the slot with the next item.
// A row always yields its near item (possibly empty), so it ends on exactly one item,
// where the lanes' sums are combined and stored. Zero-filled entries gather zg[0] with
// h = 0 and add an exact zero. Rows start on 16-byte boundaries (capacities are multiples
// of 32 entries).
// The ring holds SP_RING_SLOTS slots per block: SP_SLOTS per warp at 32 warps, twice as many
// per warp at 16 warps (the same bytes in flight per SM with half the threads).
constexpr int SP_SLOTS = 3;
constexpr int SP_RING_SLOTS = 32 * SP_SLOTS;
constexpr int SP_SLOT_BYTES = 1024;
constexpr int SP_RING_BYTES = SP_RING_SLOTS * SP_SLOT_BYTES + SP_RING_SLOTS * 4;   // slots, then tags

struct SpCursor {
  int i, part, k0;             // next item: row, part (0 near, 1 far), first entry
  int bb, bn, bf;              // rows bb..bb+31: this lane holds the counts of row bb + lane
};

__device__ __forceinline__ void sp_counts(const CG<float>& a, SpCursor& c, int whi) {
  const int i = c.bb + (threadIdx.x & 31);
  c.bn = i < whi ? __ldg(a.cntn + i) : 0;
  c.bf = i < whi ? __ldg(a.cnt + i) : 0;
}

// 16-byte copy with an L2 evict-first policy: the matrix is read once per SpMV and does not
// stay in L2 between SpMVs (126 MB L2, > 100 MB per SpMV), so it should not push out the
// gathered vector or the data of kernels running beside the solve
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16(unsigned saddr, const void* g, int nbytes, unsigned long long pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(saddr), "l"(g), "r"(nbytes),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// copies the cursor's item into the slot at shared address sa and moves the cursor to the
// next item; returns the item's tag: 2 row + 1 when the item ends its row, else 2 row
__device__ __forceinline__ int sp_issue(const CG<float>& a, SpCursor& c, int whi, unsigned sa) {
  const int lane = threadIdx.x & 31;
  const int n = __shfl_sync(0xffffffffu, c.part == 0 ? c.bn : c.bf, c.i - c.bb);
  const size_t base = c.part == 0 ? (size_t)c.i * a.capn : (size_t)c.i * a.cap;
  const int* cr = (c.part == 0 ? a.coln : a.col) + base;
  const float* hr = (c.part == 0 ? a.Hn : a.H) + base;
  const int k = c.k0 + 4 * lane;
  const int nb = k < n ? min(4 * (n - k), 16) : 0;
  const int ko = nb > 0 ? k : 0;
  const unsigned long long pol = l2_evict_first();
  cp_async16(sa + 16 * lane, cr + ko, nb, pol);
  cp_async16(sa + 512 + 16 * lane, hr + ko, nb, pol);
  const int tag = 2 * c.i;
  c.k0 += 128;
  if (c.part == 0) {
    if (c.k0 < n) return tag;
    c.part = 1;
    c.k0 = 0;
  }
  if (c.k0 < __shfl_sync(0xffffffffu, c.bf, c.i - c.bb)) return tag;
  ++c.i;
  c.part = 0;
  c.k0 = 0;
  if (c.i - c.bb == 32) {
    c.bb = c.i;
    sp_counts(a, c, whi);
  }
  return tag + 1;
}

template <int SLOTS>
__device__ __forceinline__ void spmv_ring_f(const CG<float>& a, unsigned char* ring, int wlo, int whi, float* us,
                                            float* ut) {
  static_assert(SLOTS * 32 <= SP_RING_SLOTS * 32 && SP_RING_SLOTS % SLOTS == 0, "ring slots");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float2* zg = (const float2*)a.zg;
  unsigned char* mine = ring + wid * SLOTS * SP_SLOT_BYTES;
  int* tags = (int*)(ring + SP_RING_SLOTS * SP_SLOT_BYTES) + wid * SLOTS;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(mine);
  SpCursor c;
  c.i = wlo; c.part = 0; c.k0 = 0; c.bb = wlo;
  sp_counts(a, c, whi);
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int tag = c.i < whi ? sp_issue(a, c, whi, sbase + sl * SP_SLOT_BYTES) : -1;
    if (lane == 0) tags[sl] = tag;
    cp_commit();
  }
  float sf = 0.f, tf = 0.f;
  for (int sl = 0;; sl = sl + 1 == SLOTS ? 0 : sl + 1) {
    asm volatile("cp.async.wait_group %0;" ::"n"(SLOTS - 1) : "memory");
    __syncwarp();
    const int tag = tags[sl];
    if (tag < 0) break;
    const int* sj = (const int*)(mine + sl * SP_SLOT_BYTES);
    const float* sh = (const float*)(mine + sl * SP_SLOT_BYTES + 512);
    const int j0 = sj[lane], j1 = sj[lane + 32], j2 = sj[lane + 64], j3 = sj[lane + 96];
    const float h0 = sh[lane], h1 = sh[lane + 32], h2 = sh[lane + 64], h3 = sh[lane + 96];
    const float2 z0 = zg[j0], z1 = zg[j1], z2 = zg[j2], z3 = zg[j3];
    __syncwarp();                                        // every lane has read the slot
    const int nt = c.i < whi ? sp_issue(a, c, whi, sbase + sl * SP_SLOT_BYTES) : -1;
    if (lane == 0) tags[sl] = nt;
    cp_commit();
    sf = fmaf(h0, z0.x, sf); tf = fmaf(h0, z0.y, tf);
    sf = fmaf(h1, z1.x, sf); tf = fmaf(h1, z1.y, tf);
    sf = fmaf(h2, z2.x, sf); tf = fmaf(h2, z2.y, tf);
    sf = fmaf(h3, z3.x, sf); tf = fmaf(h3, z3.y, tf);
    if (tag & 1) {
      sf = warp_sumf(sf);
      tf = warp_sumf(tf);
      if (lane == 0) { us[tag >> 1] = sf; ut[tag >> 1] = tf; }
      sf = 0.f;
      tf = 0.f;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
}

// where a block keeps its per-replica scalars and the CG vectors of its rows: shared
// memory when they fit (the host decides), else a block-private global region. Either way
// only this block reads or writes them, so no value crosses blocks except through zg and
// the chunk partials.
struct Blk {
  unsigned char* ring;         // SpMV streaming ring (mixed path)
  float* bjs;                  // this block's block-Jacobi inverses in shared memory (or null)
  double* S;                   // [nrep*NS + 4] scalars, then [nrep*NQ] reduced totals
  double* red;
  double* st;                  // [NV_STATE][rows] row state (structure of arrays)
  int rows;
  __device__ __forceinline__ double& v(int k, int li) const { return st[k * rows + li]; }
  template <typename R>
  __device__ __forceinline__ R* u(int sys) const { return (R*)(st + V_U * rows) + sys * rows; }
  // element (0, 0) of the inverse of the block holding row i (local row li), from shared
  // memory when staged there, else from global memory
  template <typename A>
  __device__ __forceinline__ const float* bj_of(const A& a, int i, int li) const {
    const int t = threadIdx.x & 31;
    return bjs ? bjs + 32 * (li - t) : a.binv + 32 * (size_t)(i - t);
  }
};

// off-diagonal SpMV of the chunk's rows into this block's U arrays (path precision). Warp w
// owns a contiguous run of rows (neighbouring atoms, so its gathers share cache lines).
template <typename R>
__device__ __forceinline__ void spmv_chunk(const CG<R>& a, const Blk& B, int lo, int hi, int off) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = (hi - lo + nw - 1) / nw;
  const int wlo = lo + wid * rpw, whi = min(hi, wlo + rpw);
  const typename G2<R>::T* zg = (const typename G2<R>::T*)a.zg;
  R* us = B.u<R>(0);
  R* ut = B.u<R>(1);
  if constexpr (sizeof(R) == 4) {
    if (wlo < whi) {
      if (nw == 8) spmv_ring_f<4 * SP_SLOTS>(a, B.ring, wlo, whi, us + off - lo, ut + off - lo);
      else if (nw == 16) spmv_ring_f<2 * SP_SLOTS>(a, B.ring, wlo, whi, us + off - lo, ut + off - lo);
      else spmv_ring_f<SP_SLOTS>(a, B.ring, wlo, whi, us + off - lo, ut + off - lo);
    }
    return;
  }
  for (int i = wlo; i < whi; ++i) {
    R sf = 0, tf = 0;
    spmv_part<R>(a.cntn, a.coln, a.Hn, a.capn, i, zg, sf, tf);
    spmv_part<R>(a.cnt, a.col, a.H, a.cap, i, zg, sf, tf);
    sf = warp_total(sf);
    tf = warp_total(tf);
    if (lane == 0) {
      us[off + i - lo] = sf;
      ut[off + i - lo] = tf;
    }
  }
}

template <typename R>
struct Chunks {
  int lo[MAXC], hi[MAXC], rep[MAXC];
};
template <typename R>
__device__ __forceinline__ void chunk_of(const CG<R>& a, const Chunks<R>& C, int k, int c, int& lo, int& hi,
                                         int& rep) {
  if (k < MAXC) {
    lo = C.lo[k]; hi = C.hi[k]; rep = C.rep[k];
  } else {
    lo = a.chunk_lo[c]; hi = a.chunk_lo[c + 1]; rep = a.chunk_rep[c];
  }
}
// f(chunk, lo, hi, rep, local offset of the chunk's first row in this block's state)
template <typename R, typename F>
__device__ __forceinline__ void for_chunks(const CG<R>& a, const Chunks<R>& C, F&& f) {
  int off = 0, k = 0;
  for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x, ++k) {
    int lo, hi, rep;
    chunk_of(a, C, k, c, lo, hi, rep);
    f(c, lo, hi, rep, off);
    off += hi - lo;
  }
}
// dense row map: thread t takes rows lo + t, lo + t + blockDim.x, ...
template <typename F>
__device__ __forceinline__ void for_rows(int lo, int hi, F&& f) {
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) f(i);
}

// warp-uniform row map (same rows per thread as for_rows): f(i, valid) on all 32 lanes of a
// warp, valid = i < hi, so warp shuffles inside f see every lane
template <typename F>
__device__ __forceinline__ void for_warp_rows(int lo, int hi, F&& f) {
  const int lane = threadIdx.x & 31;
  for (int base = lo + (int)threadIdx.x - lane; base < hi; base += blockDim.x) f(base + lane, base + lane < hi);
}

// block-Jacobi preconditioner: (zs, zt) = B^-1 (rs, rt) over the warp's block (chunks
// start on block boundaries, so a warp's rows are one block: its valid lanes, a prefix of
// nv). FP32: lane t sums B^-1[t][m] r_m over m < nv with r_m from lane m; Bc points at
// element (0, 0) of the block's column-major inverse (element (t, m) at Bc[32 m + t])
__device__ __forceinline__ void bj_apply(const float* Bc, int nv, double rs, double rt, double& zs, double& zt) {
  const int lane = threadIdx.x & 31;
  Bc += lane;
  const float fs = (float)rs, ft = (float)rt;
  float as = 0.f, at = 0.f;
#pragma unroll 8
  for (int m = 0; m < nv; ++m) {
    const float b = Bc[32 * m];
    as = fmaf(b, __shfl_sync(0xffffffffu, fs, m), as);
    at = fmaf(b, __shfl_sync(0xffffffffu, ft, m), at);
  }
  zs = (double)as;
  zt = (double)at;
}

template <typename R>
__device__ __forceinline__ void put_zg(const CG<R>& a, int i, double s, double t) {
  using T = typename G2<R>::T;
  T v;
  v.x = (R)s;
  v.y = (R)t;
  ((T*)a.zg)[i] = v;
}

// total of the active flags over replicas -> S[nrep*NS] (thread 0, after the block's
// scalar updates; fenced by __syncthreads on both sides)
__device__ __forceinline__ void count_active(double* S, int nrep) {
  __syncthreads();
  if (threadIdx.x == 0) {
    double act = 0;
    for (int r = 0; r < nrep; ++r) act += S[r * NS + S_ACT_S] + S[r * NS + S_ACT_T];
    S[nrep * NS] = act;
  }
  __syncthreads();
}

// NT threads per block, one block per SM; every loop is strided by blockDim.x. NT < 1024
// is the shape for running beside other kernels (fewer registers held per SM); the register
// budget stays 64 per thread for every NT.
template <typename R, int NT = 1024>
__global__ void __launch_bounds__(NT, 1024 / NT) k_cg(CG<R> a) {
  extern __shared__ double dsm_all[];
  __shared__ Chunks<R> C;
  Blk B;
  B.ring = (unsigned char*)dsm_all;
  double* dsm = dsm_all + a.ring_bytes / sizeof(double);
  const int sc = a.nrep * (NS + NQ) + 4;
  B.S = a.scal_smem ? dsm : a.scal + (size_t)blockIdx.x * sc;
  B.red = B.S + a.nrep * NS + 4;
  B.rows = a.rows_blk;
  B.st = a.state_smem ? dsm + (a.scal_smem ? sc : 0) : a.state + (size_t)blockIdx.x * NV_STATE * a.rows_blk;
  B.bjs = a.bj_smem ? (float*)(dsm + (a.scal_smem ? sc : 0) + (a.state_smem ? NV_STATE * a.rows_blk : 0)) : nullptr;
  for (int k = threadIdx.x; k < MAXC; k += blockDim.x) {
    const int c = blockIdx.x + k * gridDim.x;
    if (c < a.nchunk) {
      C.lo[k] = a.chunk_lo[c]; C.hi[k] = a.chunk_lo[c + 1]; C.rep[k] = a.chunk_rep[c];
    }
  }
  const bool lead = blockIdx.x == 0;
  unsigned bt = 0;                         // barriers passed x grid size
  __syncthreads();
  if (B.bjs) {
    // stage this block's inverses: row i's entries (t, m), m < its block's size
    for_chunks(a, C, [&](int, int lo, int hi, int, int off) {
      for_rows(lo, hi, [&](int i) {
        const int t = (i - lo) & 31, li = off + i - lo;
        const int nv = min(32, hi - (i - t));
        const float* g = a.binv + 32 * (size_t)(i - t) + t;
        float* d = B.bjs + 32 * (li - t) + t;
        for (int m = 0; m < nv; ++m) d[32 * m] = __ldg(g + 32 * m);
      });
    });
  }
  int pb = 0;
  double* S = B.S;
  double* red = B.red;
  const int hpos = a.hst[0], nhist = a.hst[2];
  const int nh = a.warm ? min(nhist, rx::QEQ_HIST) : 0;
  const size_t n = (size_t)a.n;
  double* outs = a.hist_s + (size_t)((hpos + 1) % rx::QEQ_HIST) * n;   // the oldest slots
  double* outt = a.hist_t + (size_t)((hpos + 1) % rx::QEQ_HIST) * n;
  // ---------------- init: eta, 1/eta and the initial guess into the row state; guess into
  // zg. Guess: x = sum_k w[p][sys][nh][k] x_k over the nh newest solutions (newest first),
  // with the host's weights of the replica's current predictor p (0 without a history)
  constexpr int H = rx::QEQ_HIST;
  auto wrow = [&](int p, int sys) { return a.wext + ((size_t)(p * 2 + sys) * (H + 1) + nh) * H; };
  __syncthreads();
  for_chunks(a, C, [&](int, int lo, int hi, int rep, int off) {
    const double* wsv = wrow(a.pred[2 * rep], 0);
    const double* wtv = wrow(a.pred[2 * rep + 1], 1);
    for_rows(lo, hi, [&](int i) {
      const int li = off + i - lo;
      const int t = a.type[i];
      double xs = 0.0, xt = 0.0;
      for (int k = 0; k < nh; ++k) {
        const size_t slot = (size_t)((hpos - k + rx::QEQ_HIST) % rx::QEQ_HIST) * n;
        xs += __ldg(wsv + k) * a.hist_s[slot + i];
        xt += __ldg(wtv + k) * a.hist_t[slot + i];
      }
      const double e = a.eta[t], ie = a.ieta[t];
      B.v(V_ETA, li) = e; B.v(V_IETA, li) = ie;
      B.v(V_XS, li) = xs; B.v(V_XT, li) = xt;
      put_zg(a, i, xs, xt);
    });
  });
  if (a.qhat && nhist > 0 && lead)
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) a.mlp_used[r] = 0;
  if (a.qhat && nhist == 0) {
    // learned guess for s (only without a usable history: with one, the extrapolated guess
    // is used and the learned one was not computed): s_mlp = q^ + mu t_ext with mu = sum
    // s_ext / sum t_ext of the replica (then s_mlp - mu t_ext = q^); kept for a replica when
    // its initial residual ||b_s - H s|| is below the extrapolated guess's (one extra SpMV
    // for both candidates)
    for_chunks(a, C, [&](int c, int lo, int hi, int, int off) {
      double v[2] = {0, 0};
      for_rows(lo, hi, [&](int i) {
        v[0] += B.v(V_XS, off + i - lo);
        v[1] += B.v(V_XT, off + i - lo);
      });
      block_sum<2>(a, v, hi - lo, pb, c);
    });
    if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
    reduce_parts<2>(a, pb, red);
    pb ^= 1;
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x)
      S[r * NS + S_MU] = red[r * NQ + 1] != 0.0 ? red[r * NQ + 0] / red[r * NQ + 1] : 0.0;
    __syncthreads();
    for_chunks(a, C, [&](int, int lo, int hi, int rep, int off) {
      const double mu = S[rep * NS + S_MU];
      for_rows(lo, hi, [&](int i) {
        const int li = off + i - lo;
        put_zg(a, i, (double)a.qhat[i] + mu * B.v(V_XT, li), B.v(V_XS, li));
      });
    });
    if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
    for_chunks(a, C, [&](int c, int lo, int hi, int rep, int off) {
      spmv_chunk(a, B, lo, hi, off);
      __syncthreads();
      const double mu = S[rep * NS + S_MU];
      const R* us = B.u<R>(0);
      const R* ut = B.u<R>(1);
      double v[2] = {0, 0};
      for_rows(lo, hi, [&](int i) {
        const int li = off + i - lo;
        const double e = B.v(V_ETA, li), bs = -a.chi[a.type[i]];
        const double sm = (double)a.qhat[i] + mu * B.v(V_XT, li);
        const double r1 = bs - ((double)us[li] + e * sm), r2 = bs - ((double)ut[li] + e * B.v(V_XS, li));
        v[0] += r1 * r1;
        v[1] += r2 * r2;
      });
      block_sum<2>(a, v, hi - lo, pb, c);
    });
    if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
    reduce_parts<2>(a, pb, red);
    pb ^= 1;
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
      const bool use = red[r * NQ + 0] < red[r * NQ + 1];
      S[r * NS + S_USE] = use ? 1.0 : 0.0;
      if (lead) a.mlp_used[r] = use ? 1 : 0;
    }
    __syncthreads();
    for_chunks(a, C, [&](int, int lo, int hi, int rep, int off) {
      const bool use = S[rep * NS + S_USE] > 0.0;
      const double mu = S[rep * NS + S_MU];
      for_rows(lo, hi, [&](int i) {
        const int li = off + i - lo;
        if (use) B.v(V_XS, li) = (double)a.qhat[i] + mu * B.v(V_XT, li);
        put_zg(a, i, B.v(V_XS, li), B.v(V_XT, li));
      });
    });
  }
  if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
  // r = b - H x, z = M^-1 r, p = w = 0
  for_chunks(a, C, [&](int c, int lo, int hi, int, int off) {
    spmv_chunk(a, B, lo, hi, off);
    __syncthreads();
    double v[6] = {0, 0, 0, 0, 0, 0};
    const R* us = B.u<R>(0);
    const R* ut = B.u<R>(1);
    auto resid = [&](int i, int li, double& rs, double& rt) {
      const double e = B.v(V_ETA, li);
      const double hs = (double)us[li] + e * B.v(V_XS, li);
      const double ht = (double)ut[li] + e * B.v(V_XT, li);
      const double bs = -a.chi[a.type[i]], bt = -1.0;
      rs = bs - hs; rt = bt - ht;
      B.v(V_RS, li) = rs; B.v(V_RT, li) = rt;
      B.v(V_PS, li) = 0; B.v(V_PT, li) = 0; B.v(V_WS, li) = 0; B.v(V_WT, li) = 0;
      v[2] += rs * rs; v[3] += rt * rt;             // r.r
      v[4] += bs * bs; v[5] += bt * bt;             // b.b
    };
    if (a.binv) {
      for_warp_rows(lo, hi, [&](int i, bool valid) {
        const int li = off + i - lo;
        double rs = 0.0, rt = 0.0, zs, zt;
        if (valid) resid(i, li, rs, rt);
        bj_apply(B.bj_of(a, i, li), __popc(__ballot_sync(0xffffffffu, valid)), rs, rt, zs, zt);
        if (valid) {
          B.v(V_ZS, li) = zs; B.v(V_ZT, li) = zt;
          v[0] += rs * zs; v[1] += rt * zt;         // r.z
        }
      });
    } else {
      for_rows(lo, hi, [&](int i) {
        const int li = off + i - lo;
        const double ie = B.v(V_IETA, li);
        double rs, rt;
        resid(i, li, rs, rt);
        B.v(V_ZS, li) = rs * ie; B.v(V_ZT, li) = rt * ie;
        v[0] += rs * rs * ie; v[1] += rt * rt * ie; // r.z
      });
    }
    block_sum<6>(a, v, hi - lo, pb, c);
  });
  if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
  reduce_parts<6>(a, pb, red);
  pb ^= 1;
  for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
    double* sr = S + r * NS;
    const double* rd = red + r * NQ;
    sr[S_RHO_S] = rd[0]; sr[S_RHO_T] = rd[1];
    sr[S_BB_S] = rd[4]; sr[S_BB_T] = rd[5];
    sr[S_BE_S] = 0; sr[S_BE_T] = 0;
    sr[S_ACT_S] = rd[2] > a.tol2 * rd[4] ? 1.0 : 0.0;
    sr[S_ACT_T] = rd[3] > a.tol2 * rd[5] ? 1.0 : 0.0;
    if (lead) { a.iters[2 * r] = 0; a.iters[2 * r + 1] = 0; }
  }
  if (lead && threadIdx.x == 0) *a.spmv_total += 1;   // the initial residual
  count_active(S, a.nrep);
  // z into zg for the first iteration's SpMV: every block has finished the initial SpMV
  // (which gathered x from the same buffer) -- the barrier above -- and the next barrier
  // publishes it
  for_chunks(a, C, [&](int, int lo, int hi, int, int off) {
    for_rows(lo, hi, [&](int i) {
      const int li = off + i - lo;
      put_zg(a, i, B.v(V_ZS, li), B.v(V_ZT, li));
    });
  });
  if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
  int it = 0;
  while (S[a.nrep * NS] > 0.0 && it < a.max_iter) {
    ++it;
    // ---------------- A: u = H z; p = z + beta p; w = u + beta w; p.w
    for_chunks(a, C, [&](int c, int lo, int hi, int rep, int off) {
      spmv_chunk(a, B, lo, hi, off);
      __syncthreads();
      const double* sr = S + rep * NS;
      const bool as = sr[S_ACT_S] > 0, at = sr[S_ACT_T] > 0;
      const double bes = sr[S_BE_S], bet = sr[S_BE_T];
      const R* us = B.u<R>(0);
      const R* ut = B.u<R>(1);
      double v[2] = {0, 0};
      for_rows(lo, hi, [&](int i) {
        const int li = off + i - lo;
        const double e = B.v(V_ETA, li);
        if (as) {
          const double z = B.v(V_ZS, li);
          const double p = z + bes * B.v(V_PS, li), w = (double)us[li] + e * z + bes * B.v(V_WS, li);
          B.v(V_PS, li) = p; B.v(V_WS, li) = w; v[0] += p * w;
        }
        if (at) {
          const double z = B.v(V_ZT, li);
          const double p = z + bet * B.v(V_PT, li), w = (double)ut[li] + e * z + bet * B.v(V_WT, li);
          B.v(V_PT, li) = p; B.v(V_WT, li) = w; v[1] += p * w;
        }
      });
      block_sum<2>(a, v, hi - lo, pb, c);
    });
    if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
    reduce_parts<2>(a, pb, red);
    pb ^= 1;
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
      double* sr = S + r * NS;
      sr[S_AL_S] = sr[S_ACT_S] > 0 ? sr[S_RHO_S] / red[r * NQ + 0] : 0.0;
      sr[S_AL_T] = sr[S_ACT_T] > 0 ? sr[S_RHO_T] / red[r * NQ + 1] : 0.0;
    }
    __syncthreads();
    // ---------------- B: x += alpha p; r -= alpha w; z = r / eta; r.z, r.r
    for_chunks(a, C, [&](int c, int lo, int hi, int rep, int off) {
      const double* sr = S + rep * NS;
      const bool as = sr[S_ACT_S] > 0, at = sr[S_ACT_T] > 0;
      const double als = sr[S_AL_S], alt = sr[S_AL_T];
      double v[4] = {0, 0, 0, 0};
      if (a.binv) {
        for_warp_rows(lo, hi, [&](int i, bool valid) {
          const int li = off + i - lo;
          double rs = 0.0, rt = 0.0;
          if (valid) {
            if (as) {
              B.v(V_XS, li) += als * B.v(V_PS, li);
              rs = B.v(V_RS, li) - als * B.v(V_WS, li);
              B.v(V_RS, li) = rs;
              v[2] += rs * rs;
            }
            if (at) {
              B.v(V_XT, li) += alt * B.v(V_PT, li);
              rt = B.v(V_RT, li) - alt * B.v(V_WT, li);
              B.v(V_RT, li) = rt;
              v[3] += rt * rt;
            }
          }
          double zs, zt;
          bj_apply(B.bj_of(a, i, li), __popc(__ballot_sync(0xffffffffu, valid)), rs, rt, zs, zt);
          if (valid) {
            if (as) { B.v(V_ZS, li) = zs; v[0] += rs * zs; } else zs = B.v(V_ZS, li);
            if (at) { B.v(V_ZT, li) = zt; v[1] += rt * zt; } else zt = B.v(V_ZT, li);
            put_zg(a, i, zs, zt);
          }
        });
      } else {
        for_rows(lo, hi, [&](int i) {
          const int li = off + i - lo;
          const double ie = B.v(V_IETA, li);
          double zs = B.v(V_ZS, li), zt = B.v(V_ZT, li);
          if (as) {
            B.v(V_XS, li) += als * B.v(V_PS, li);
            const double r = B.v(V_RS, li) - als * B.v(V_WS, li);
            zs = r * ie;
            B.v(V_RS, li) = r; B.v(V_ZS, li) = zs;
            v[0] += r * zs; v[2] += r * r;
          }
          if (at) {
            B.v(V_XT, li) += alt * B.v(V_PT, li);
            const double r = B.v(V_RT, li) - alt * B.v(V_WT, li);
            zt = r * ie;
            B.v(V_RT, li) = r; B.v(V_ZT, li) = zt;
            v[1] += r * zt; v[3] += r * r;
          }
          put_zg(a, i, zs, zt);
        });
      }
      block_sum<4>(a, v, hi - lo, pb, c);
    });
    if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
    reduce_parts<4>(a, pb, red);
    pb ^= 1;
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
      double* sr = S + r * NS;
      if (sr[S_ACT_S] > 0) {
        if (lead) a.iters[2 * r] += 1;
        sr[S_BE_S] = red[r * NQ + 0] / sr[S_RHO_S];
        sr[S_RHO_S] = red[r * NQ + 0];
        if (!(red[r * NQ + 2] > a.tol2 * sr[S_BB_S])) sr[S_ACT_S] = 0.0;
      }
      if (sr[S_ACT_T] > 0) {
        if (lead) a.iters[2 * r + 1] += 1;
        sr[S_BE_T] = red[r * NQ + 1] / sr[S_RHO_T];
        sr[S_RHO_T] = red[r * NQ + 1];
        if (!(red[r * NQ + 3] > a.tol2 * sr[S_BB_T])) sr[S_ACT_T] = 0.0;
      }
    }
    if (lead && threadIdx.x == 0) *a.spmv_total += 1;
    count_active(S, a.nrep);
  }
  if (S[a.nrep * NS] > 0.0 && lead && threadIdx.x == 0) atomicOr(a.err, ERR_CG);
  // ---------------- solutions out; mu = sum s / sum t per replica, q = s - mu t. With an
  // adaptive guess, also the squared error every predictor's guess would have had for this
  // solve (same history), so that each replica and system uses the best one next time
  const bool score = a.adapt && nh > 0;
  for_chunks(a, C, [&](int c, int lo, int hi, int, int off) {
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // sum s, sum t, error of s by predictor 0..2, of t
    for_rows(lo, hi, [&](int i) {
      const int li = off + i - lo;
      const double xs = B.v(V_XS, li), xt = B.v(V_XT, li);
      if (score) {
#pragma unroll
        for (int p = 0; p < rx::QEQ_NPRED; ++p) {
          const double* ws = wrow(p, 0);
          const double* wt = wrow(p, 1);
          double gs = 0.0, gt = 0.0;
          for (int k = 0; k < nh; ++k) {
            const size_t slot = (size_t)((hpos - k + H) % H) * n;
            gs += __ldg(ws + k) * a.hist_s[slot + i];
            gt += __ldg(wt + k) * a.hist_t[slot + i];
          }
          v[2 + p] += (gs - xs) * (gs - xs);
          v[5 + p] += (gt - xt) * (gt - xt);
        }
      }
      outs[i] = xs;                          // after the history was read: this is its oldest slot
      outt[i] = xt;
      v[0] += xs;
      v[1] += xt;
    });
    block_sum<8>(a, v, hi - lo, pb, c);
  });
  if (!grid_barrier(a.bar, a.err, bt, a.bar_limit)) return;
  reduce_parts<8>(a, pb, red);
  for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
    const double* rd = red + r * NQ;
    S[r * NS + S_MU] = rd[0] / rd[1];
    if (score && lead) {
      int bs = 0, bt2 = 0;
      for (int p = 1; p < rx::QEQ_NPRED; ++p) {
        if (rd[2 + p] < rd[2 + bs]) bs = p;
        if (rd[5 + p] < rd[5 + bt2]) bt2 = p;
      }
      a.pred[2 * r] = bs;
      a.pred[2 * r + 1] = bt2;
    }
  }
  __syncthreads();
  for_chunks(a, C, [&](int, int lo, int hi, int rep, int off) {
    const double mu = S[rep * NS + S_MU];
    for_rows(lo, hi, [&](int i) {
      const int li = off + i - lo;
      const double qi = B.v(V_XS, li) - mu * B.v(V_XT, li);
      a.q[i] = qi;
      a.qf[i] = (float)qi;
      if (a.ph) ((float*)(a.ph + i))[3] = (float)qi;
    });
  });
  // advance the history (every block read hst before its first barrier)
  if (lead && threadIdx.x == 0) {
    a.hst[0] = (hpos + 1) % rx::QEQ_HIST;
    a.hst[1] = a.hst[0];
    a.hst[2] = nhist < rx::QEQ_HIST ? nhist + 1 : rx::QEQ_HIST;
  }
}


// Block-Jacobi setup: one warp per block of sz <= 32 consecutive atoms (b0..b0+sz-1) of one
// replica. The block's H in shared memory: eta on the diagonal and, for a != b, the sum over
// every image of atom b within r_nb of Tap(r) k_e (r^3 + gamma^-3)^(-1/3) (the image vector
// from the float hi/lo positions, exact to ~1 ulp; an image decided the other way at r_nb
// carries a vanishing taper), each unordered pair evaluated once; rows and columns past sz
// the identity's. The block is a principal submatrix of H, so symmetric positive definite:
// Gauss-Jordan without pivoting inverts it in registers (row a in lane a, the pivot row by
// shuffles), and the inverse, symmetrised, is stored column by column.
constexpr int BJ_WARPS = 4;

__global__ void __launch_bounds__(BJ_WARPS * 32) k_bj_build(Sys s, const DParams<float>* __restrict__ P,
                                                            const int* __restrict__ bstart,
                                                            const int* __restrict__ bsize, int nblk,
                                                            float* __restrict__ binv) {
  __shared__ float T[BJ_WARPS][32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int blk = blockIdx.x * BJ_WARPS + w;
  if (blk >= nblk) return;                              // whole warps
  const int b0 = bstart[blk], sz = bsize[blk];
  float* Trow = T[w][lane];
  for (int b = 0; b < 32; ++b) Trow[b] = b == lane ? 1.0f : 0.0f;
  if (lane < sz) Trow[lane] = P->eta[s.type[b0 + lane]];
  __syncwarp();
  // each unordered pair {a, b} once: lane a takes b = a + d (mod 32), d = 1..15, and lanes
  // below 16 also d = 16 (15 or 16 pairs a lane); the value goes to both (a, b) and (b, a)
  {
    const int a = lane;
    const float rnb = P->r_nb, rnb2 = rnb * rnb, ke = P->k_e;
    const int ia = b0 + a;
    const int rp = s.rep[b0];
    const float Lh[3] = {s.boxh[3 * rp], s.boxh[3 * rp + 1], s.boxh[3 * rp + 2]};
    const float Ll[3] = {s.boxl[3 * rp], s.boxl[3 * rp + 1], s.boxl[3 * rp + 2]};
    float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
    int ta = 0;
    if (a < sz) {
      ah[0] = s.xh[ia]; ah[1] = s.yh[ia]; ah[2] = s.zh[ia];
      al[0] = s.xl[ia]; al[1] = s.yl[ia]; al[2] = s.zl[ia];
      ta = s.type[ia];
    }
    const int dmax = a < 16 ? 16 : 15;
#pragma unroll 1
    for (int d = 1; d <= dmax; ++d) {
      const int b = (a + d) & 31;
      if (a >= sz || b >= sz) continue;
      const int ib = b0 + b;
      const float bh[3] = {s.xh[ib], s.yh[ib], s.zh[ib]}, bl[3] = {s.xl[ib], s.yl[ib], s.zl[ib]};
      const float g = P->gamma_m3[ta * MAXT + s.type[ib]];
      // per dimension the image shifts within r_nb: at most two, the box exceeding r_nb
      float d0[3], d1[3];
      int nv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        nv[c] = 0;
        d0[c] = d1[c] = 0.f;
#pragma unroll
        for (int sh = -1; sh <= 1; ++sh) {
          const float v = pv_comp(bh[c], ah[c], bl[c], al[c], sh, Lh[c], Ll[c]);
          if (fabsf(v) < rnb) {
            if (nv[c] == 0) d0[c] = v; else d1[c] = v;
            ++nv[c];
          }
        }
      }
      float h = 0.f;
#pragma unroll 1
      for (int x = 0; x < nv[0]; ++x)
#pragma unroll 1
        for (int y = 0; y < nv[1]; ++y)
#pragma unroll 1
          for (int z = 0; z < nv[2]; ++z) {
            const float dx = x ? d1[0] : d0[0], dy = y ? d1[1] : d0[1], dz = z ? d1[2] : d0[2];
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rnb2) {
              const float rr = sqrtf(r2);
              float tap, dtap;
              taper<float>(rr, rnb, tap, dtap);
              h += tap * ke * rcbrtf(rr * rr * rr + g);
            }
          }
      T[w][a][b] = h;
      T[w][b][a] = h;
    }
  }
  __syncwarp();
  float R[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) R[b] = Trow[b];
  __syncwarp();
  // Gauss-Jordan: after step k, column k holds the inverse's column k
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float ip = 1.0f / __shfl_sync(0xffffffffu, R[k], k);
    const float f = R[k] * ip;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float rkj = __shfl_sync(0xffffffffu, R[j], k);
      if (lane == k) R[j] = j == k ? ip : rkj * ip;
      else R[j] = j == k ? -f : fmaf(-f, rkj, R[j]);
    }
  }
#pragma unroll
  for (int m = 0; m < 32; ++m) T[w][lane][m] = R[m];
  __syncwarp();
  // columns m < sz only: a shorter block ends where the next replica's first block begins
  float* out = binv + 32 * (size_t)b0 + lane;
  for (int m = 0; m < sz; ++m) out[32 * m] = 0.5f * (T[w][lane][m] + T[w][m][lane]);
}

}  // namespace

namespace rx {

template <typename R>
int qeq_solve(const Launch& L, Sys s, FarList f, QeqState& Q, const DParams<R>* P, const double* chi,
              const double* eta, double tol, int max_iter, int warm, const float* qhat, int threads,
              int layout) {
  (void)P;
  if (layout < 0 || layout >= QEQ_NLAYOUT || (layout > 0 && threads != 1024)) return -1;
  const QeqLayout& Y = Q.lay[layout];
  CG<R> a;
  a.n = s.n; a.nrep = s.nrep; a.nchunk = Y.nchunk; a.max_iter = max_iter;
  a.tol2 = tol * tol;
  a.type = s.type;
  a.cnt = f.cnt; a.col = f.j; a.H = (const R*)f.H; a.cap = f.cap;
  a.cntn = f.cntn; a.coln = f.jn; a.Hn = (const R*)f.Hn; a.capn = f.capn;
  a.eta = eta; a.chi = chi;
  a.binv = Q.precond == REAXFF_PRECOND_BLOCK32 ? Q.binv : nullptr;
  a.bj_smem = a.binv ? Y.bj_smem : 0;
  a.hist_s = Q.hist_s; a.hist_t = Q.hist_t; a.hst = Q.hst; a.wext = Q.wext; a.pred = Q.pred;
  a.adapt = warm != REAXFF_WARM_LAGRANGE;
  a.warm = (warm == REAXFF_WARM_EXTRAP || warm == REAXFF_WARM_MLP || warm == REAXFF_WARM_LAGRANGE) ? 1 : 0;
  a.qhat = qhat;
  a.mlp_used = Q.mlp_used;
  a.zg = Q.zg;
  a.q = s.q; a.qf = s.qf; a.ph = s.ph; a.part = Q.part; a.scal = Q.scal; a.state = Q.state;
  a.rows_blk = Y.rows_blk; a.scal_smem = Y.scal_smem; a.state_smem = Y.state_smem;
  a.ring_bytes = Q.ring_bytes;
  a.ieta = Q.ieta;
  a.chunk_lo = Y.chunk_lo; a.chunk_rep = Y.chunk_rep; a.rep_chunk = Y.rep_chunk;
  a.iters = Q.iters; a.spmv_total = Q.spmv_total; a.bar = Q.bar; a.err = s.err;
  a.bar_limit = Q.bar_limit > 0 ? Q.bar_limit : BAR_CYCLE_LIMIT;
  cudaMemsetAsync(Q.bar, 0, sizeof(GridBar), L.st);
  void* args[] = {&a};
  // 1024 threads per SM, or 512 / 256 (mixed path) to leave registers and shared memory of
  // each SM to kernels running beside the solve; the shapes past the first put 1024-thread
  // blocks on a part of the SMs instead
  void* fn = (void*)k_cg<R, 1024>;
  int nt = 1024;
  if constexpr (sizeof(R) == 4) {
    if (threads == 512) { fn = (void*)k_cg<R, 512>; nt = 512; }
    else if (threads == 256) { fn = (void*)k_cg<R, 256>; nt = 256; }
  }
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(Y.grid), dim3(nt), args, Y.smem_bytes, L.st);
  *L.count += 2;
  return e == cudaSuccess ? 0 : -1;
}

int qeq_ring_bytes(bool fp64) { return fp64 ? 0 : SP_RING_BYTES; }

void qeq_precond_build(const Launch& L, Sys s, QeqState& Q) {
  if (Q.precond != REAXFF_PRECOND_BLOCK32 || Q.bj_nblk == 0) return;
  k_bj_build<<<(Q.bj_nblk + BJ_WARPS - 1) / BJ_WARPS, BJ_WARPS * 32, 0, L.st>>>(s, Q.Pf, Q.bj_start, Q.bj_size,
                                                                               Q.bj_nblk, Q.binv);
  *L.count += 1;
}

int qeq_grid_size(int nsm) {
  cudaFuncSetAttribute((const void*)k_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, QEQ_SMEM_MAX);
  cudaFuncSetAttribute((const void*)k_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, QEQ_SMEM_MAX);
  // the shapes that run beside other kernels prefer a 164 KB shared-memory carveout (72 % of
  // the maximum): an SM holding a solve block (~130 KB) keeps room for the other kernels'
  // shared memory and still 92 KB of L1 for the solve's gathers
  for (const void* f : {(const void*)k_cg<float, 512>, (const void*)k_cg<float, 256>}) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, QEQ_SMEM_MAX);
    cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 72);
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_cg<double>, 1024, QEQ_SMEM_MAX);
  int per_f = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, (const void*)k_cg<float>, 1024, QEQ_SMEM_MAX);
  if (per_f < per) per = per_f;
  if (per < 1) per = 1;
  return nsm * per;
}

template int qeq_solve<double>(const Launch&, Sys, FarList, QeqState&, const DParams<double>*, const double*,
                               const double*, double, int, int, const float*, int, int);
template int qeq_solve<float>(const Launch&, Sys, FarList, QeqState&, const DParams<float>*, const double*,
                              const double*, double, int, int, const float*, int, int);
}  // namespace rx

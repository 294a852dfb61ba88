// (f) dE/dBO chain rule into atom forces, force finalisation, energy/virial
// reductions and velocity Verlet.
//
// Paper: Table 2 "Aggregate Forces" (bond-order derivatives turned into atom forces),
// Sec. 3.1 (energies reduced system-wide, forces summed per atom; data privatisation
// replaced here by owner-computes), Sec. 4.1 (velocity-Verlet MD, dt = 0.1 fs).
//
// Chain rule (per bond, totals over both directed entries; BO, BO_pi, BO_pp are
// functions of BO' = BO'sig + BO'pi + BO'pp, BO'pi, BO'pp, Delta'_i and Delta'_j):
//   C   = dE/dBO (both entries) + dE/dsumBO_i + dE/dsumBO_j,  C_pi, C_pp likewise
//   dE/dBO'      = C (F + BO' dF/dBO') + (C_pi BO'pi + C_pp BO'pp) dG/dBO'
//   dE/dBO'pi    = C_pi G,   dE/dBO'pp = C_pp G        (F = f1 f4 f5, G = f1^2 f4 f5)
//   A_i          = sum over i's bonds of dE/dDelta'_i
//   dE/dr_ij     = (dE/dBO' + A_i + A_j) dBO'/dr + dE/dBO'pi dBO'pi/dr + dE/dBO'pp dBO'pp/dr
// One thread per unordered bond (the canonical entry e of atom i and its mirror m in atom j's
// row) in both passes. Everything above except the A_i, A_j terms is symmetric in the two
// entries (their stored factors are the same values in swapped roles), so it is evaluated
// once per bond. Pass 1 forms the three coefficients and each entry's dE/dDelta' term, from
// that entry's own stored factors, and adds the latter to A_i and A_j. Pass 2 turns the
// coefficients into the pair force, +f on i and -f on j, and the bond's virial. Per-atom sums
// (A, forces, virial) are 2^-32 fixed-point atomics: exact, so the result does not depend on
// the order of the canonical list (filled by an atomic append) or of the additions.
#include "reax_internal.cuh"

namespace {

inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }

__global__ void k_chain1(Sys s, BondList bl, AtomQ aq) {
  const int nc = *bl.ncanon;
  const double* BOp = bl.bop;
  const double* BOpi = bl.bopi;
  const double* BOpp = bl.bopp;
  const double* F1 = (const double*)bl.f1; const double* FO = (const double*)bl.fo;
  const double* FT = (const double*)bl.ft; const double* DF1 = (const double*)bl.df1;
  const double* DFOB = (const double*)bl.dfo_bo; const double* DFTB = (const double*)bl.dft_bo;
  const double* DFOD = (const double*)bl.dfo_d;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
    const int e = bl.canon[t];
    const int i = e / bl.cap;
    const int m = bl.mirror[e];
    const int j = bl.j[e];
    // exact integer sums: the same from either entry
    const double C = (double)((long long)bl.cdbo[e] + (long long)bl.cdbo[m] + (long long)aq.cddelta[i] +
                              (long long)aq.cddelta[j]) * FIX_INV;
    const double Cpi = (double)((long long)bl.cdbopi[e] + (long long)bl.cdbopi[m]) * FIX_INV;
    const double Cpp = (double)((long long)bl.cdbopp[e] + (long long)bl.cdbopp[m]) * FIX_INV;
    const double bp = BOp[e], bpi = BOpi[e], bpp = BOpp[e];
    // e is the canonical (lower) entry: its own factor f4/f5 comes first
    const double f1 = F1[e], flo = FO[e], fhi = FT[e];
    const double dflo = DFOB[e], dfhi = DFTB[e];
    const double F = f1 * flo * fhi;
    const double G = f1 * f1 * flo * fhi;
    const double d45 = dflo * fhi + flo * dfhi;
    const double dFdB = f1 * d45, dGdB = f1 * f1 * d45;
    const double piw = Cpi * bpi + Cpp * bpp;
    bl.dEdBOp[t] = C * (F + bp * dFdB) + piw * dGdB;
    bl.dEdBOpi[t] = Cpi * G;
    bl.dEdBOpp[t] = Cpp * G;
    // dE/dDelta' of each entry's own atom, from that entry's factors (own f4 first)
    {
      const double fo = FO[e], ft = FT[e], df1 = DF1[e], dfo_d = DFOD[e];
      const double dFdD = df1 * fo * ft + f1 * dfo_d * ft;
      const double dGdD = 2.0 * f1 * df1 * fo * ft + f1 * f1 * dfo_d * ft;
      fix_add(aq.A + i, C * bp * dFdD + piw * dGdD, s.err);
    }
    {
      const double f1m = F1[m], fo = FO[m], ft = FT[m], df1 = DF1[m], dfo_d = DFOD[m];
      const double dFdD = df1 * fo * ft + f1m * dfo_d * ft;
      const double dGdD = 2.0 * f1m * df1 * fo * ft + f1m * f1m * dfo_d * ft;
      fix_add(aq.A + j, C * bp * dFdD + piw * dGdD, s.err);
    }
  }
}

// pass 2: dE/dr of the bond; the pair force f = c d / r (d the entry's image vector) is
// added to i and subtracted from j, the virial -f d (both entries' halves) to atom i. Mixed
// path: c in FP64, then the force and virial products in FP32 (the precision of every other
// mixed-path force term) into the fixed-point sums
template <typename R>
__global__ void k_chain2(Sys s, BondList bl, AtomQ aq, Accum acc) {
  const int nc = *bl.ncanon;
  const R* DX = (const R*)bl.dx; const R* DY = (const R*)bl.dy; const R* DZ = (const R*)bl.dz;
  const R* RR = (const R*)bl.r;
  const double* DB = bl.dbop; const double* DBPI = bl.dbopi; const double* DBPP = bl.dbopp;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
    const int e = bl.canon[t];
    const int i = e / bl.cap;
    const int j = bl.j[e];
    const double Asum = fix_get(aq.A + i) + fix_get(aq.A + j);
    const double c = (bl.dEdBOp[t] + Asum) * DB[e] + bl.dEdBOpi[t] * DBPI[e] + bl.dEdBOpp[t] * DBPP[e];
    R cr;
    if constexpr (sizeof(R) == 4) cr = (float)(c * (double)(1.0f / RR[e]));   // FP32 reciprocal: no FP64 division
    else cr = c / (double)RR[e];
    const R dx = DX[e], dy = DY[e], dz = DZ[e];
    const R fx = cr * dx, fy = cr * dy, fz = cr * dz;
    fix_add(s.fx + i, fx, s.err);
    fix_add(s.fy + i, fy, s.err);
    fix_add(s.fz + i, fz, s.err);
    fix_add(s.fx + j, -fx, s.err);
    fix_add(s.fy + j, -fy, s.err);
    fix_add(s.fz + j, -fz, s.err);
    unsigned long long* w = acc.vfx + i;
    const size_t n = s.n;
    fix_add(w, -fx * dx, s.err);
    fix_add(w + n, -fy * dy, s.err);
    fix_add(w + 2 * n, -fz * dz, s.err);
    fix_add(w + 3 * n, -fx * dy, s.err);
    fix_add(w + 4 * n, -fx * dz, s.err);
    fix_add(w + 5 * n, -fy * dz, s.err);
  }
}

__global__ void k_finalize(Sys s, double* F) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  F[3 * i + 0] = fix_get(s.fx + i);
  F[3 * i + 1] = fix_get(s.fy + i);
  F[3 * i + 2] = fix_get(s.fz + i);
}

// Per-replica sums of the 13 energy terms, 6 virial components and the kinetic energy
// (NQ_RED quantities): pass 1, block (chunk, q) sums one chunk of <= RED_CHUNK atoms of one
// replica; pass 2, one warp per (replica, q) sums that replica's chunk partials in order.
// Both passes have a fixed reduction order, so the sums are bitwise reproducible.
constexpr int NQ_RED = NTERMS + 7;
constexpr int RED_PER_THREAD = 4, RED_BLOCK = 128;
static_assert(RED_PER_THREAD * RED_BLOCK == rx::RED_CHUNK, "reduction chunk");
__device__ __forceinline__ double red_value(const Sys& s, const Accum& acc, const double* mass_t, int q, int64_t i) {
  if (q < NTERMS) return acc.e[(size_t)q * s.n + i] + fix_get(acc.efx + (size_t)q * s.n + i);
  if (q < NTERMS + 6)
    return acc.vir[(size_t)(q - NTERMS) * s.n + i] + fix_get(acc.vfx + (size_t)(q - NTERMS) * s.n + i);
  const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
  return (vx * vx + vy * vy + vz * vz) * mass_t[s.type[i]] * (0.5 / 4.184e-4);   // (amu A^2/fs^2 -> kcal/mol)
}
// Pass 1 per block (chunk, q). Arrival counters (each zeroed again by the block that
// consumes it) then finish the sums where the data is complete: the last chunk block of a
// (replica, q) sums that replica's chunk partials of q (lane l of warp 0 takes chunks l,
// l+32, ... in order); the last of a replica's NQ_RED finishers writes its total energy
// (when asked); the last replica advances *etot_idx. The order of every sum is fixed
// whichever block comes last, and the finishing work is spread over (replica, q) pairs.
__global__ void k_reduce(Sys s, Accum acc, const double* mass_t, rx::RedPlan rp, double* E_rep, double* vir_rep,
                         double* ke_rep, double* etot, int* etot_idx) {
  const int c = blockIdx.x, q = blockIdx.y;
  // a chunk holds at most RED_PER_THREAD * blockDim.x atoms: each thread's values load
  // together and are summed in a fixed order
  const int lo = rp.chunk_lo[c], hi = rp.chunk_lo[c + 1];
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < RED_PER_THREAD; ++k) {
    const int i = lo + threadIdx.x + k * blockDim.x;
    if (i < hi) v += red_value(s, acc, mass_t, q, i);
  }
  __shared__ double sh[32];
  __shared__ int stage;          // 1: this block finishes (r, q); 2: also replica r; 3: also the launch
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  const int r = rp.chunk_rep[c];
  const int c0 = rp.rep_chunk[r], c1 = rp.rep_chunk[r + 1];
  unsigned* cnt_q = rp.done + (size_t)r * NQ_RED + q;
  unsigned* cnt_r = rp.done + (size_t)s.nrep * NQ_RED + r;
  unsigned* cnt_all = rp.done + (size_t)s.nrep * (NQ_RED + 1);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    rp.part[(size_t)c * NQ_RED + q] = t;
    __threadfence();
    stage = atomicAdd(cnt_q, 1u) == (unsigned)(c1 - c0 - 1) ? 1 : 0;
  }
  __syncthreads();
  if (stage == 0) return;
  __threadfence();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double u = 0.0;
    for (int k = c0 + lane; k < c1; k += 32) u += __ldcg(rp.part + (size_t)k * NQ_RED + q);
    u = warp_sum(u);
    if (lane == 0) {
      if (!isfinite(u)) atomicOr(s.err, ERR_NAN);
      if (q < NTERMS) E_rep[r * NTERMS + q] = u;
      else if (q < NTERMS + 6) vir_rep[r * 6 + (q - NTERMS)] = u;
      else ke_rep[r] = u;
      *cnt_q = 0u;
      __threadfence();
      stage = atomicAdd(cnt_r, 1u) == (unsigned)(NQ_RED - 1) ? 2 : 1;
    }
  }
  __syncthreads();
  if (stage < 2) return;
  if (threadIdx.x == 0) {
    __threadfence();
    if (etot) {
      // total energy of replica r into etot[k*nrep + r]; k = *etot_idx (advanced below) or 0
      const int k = etot_idx ? *etot_idx : 0;
      double t = 0.0;
      for (int qq = 0; qq < NTERMS; ++qq) t += __ldcg(E_rep + r * NTERMS + qq);
      etot[(size_t)k * s.nrep + r] = t + __ldcg(ke_rep + r);
    }
    *cnt_r = 0u;
    __threadfence();
    if (atomicAdd(cnt_all, 1u) == (unsigned)(s.nrep - 1)) {
      if (etot && etot_idx) *etot_idx += 1;
      *cnt_all = 0u;
    }
  }
}

// half kick (and drift). With skin: after the drift, also the float position records and
// the Verlet-skin test of the candidate list (displacement since the last build against
// skin/2), which the list build would otherwise do in two more passes
__global__ void k_kick_drift(Sys s, const double* mass_t, double dt, int drift, int skin, double half_skin2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double c = (0.5 * dt * 4.184e-4) * mass_t[MAXT + s.type[i]];    // mass_t[MAXT + t] = 1 / m_t
  double vx = s.vx[i] + c * fix_get(s.fx + i);
  double vy = s.vy[i] + c * fix_get(s.fy + i);
  double vz = s.vz[i] + c * fix_get(s.fz + i);
  s.vx[i] = vx; s.vy[i] = vy; s.vz[i] = vz;
  if (drift) {
    const double* L = s.box + 3 * s.rep[i];
    // x + dt v with the product and the sum rounded separately (no fused multiply-add),
    // so that a host reproduces the drift bit for bit
    double p[3] = {__dadd_rn(s.x[i], __dmul_rn(dt, vx)), __dadd_rn(s.y[i], __dmul_rn(dt, vy)),
                   __dadd_rn(s.z[i], __dmul_rn(dt, vz))};
    for (int d = 0; d < 3; ++d) {
      if (p[d] < 0.0) { p[d] += L[d]; s.img[3 * i + d] -= 1; }
      if (p[d] >= L[d]) { p[d] -= L[d]; s.img[3 * i + d] += 1; }
    }
    if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) atomicOr(s.err, ERR_NAN);
    s.x[i] = p[0]; s.y[i] = p[1]; s.z[i] = p[2];
    if (skin) {
      write_pos_f32(s, i);
      double d2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double dd = (p[d] + s.img[3 * i + d] * L[d]) - s.xb[3 * i + d];
        d2 += dd * dd;
      }
      if (!(d2 <= half_skin2)) atomicOr(s.rebuild, 1);
    }
  }
}

// copy (save) or restore the primary MD state of a batch: positions, velocities and the
// QEq solution rings with their state
__global__ void k_snapshot(Sys s, double* hist, int nhist_doubles, int* hst, double* buf, int* ibuf, int restore) {
  const size_t n = (size_t)s.n;
  double* src[6] = {s.x, s.y, s.z, s.vx, s.vy, s.vz};
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 6 * n + (size_t)nhist_doubles;
       t += (size_t)gridDim.x * blockDim.x) {
    double* p = t < 6 * n ? src[t / n] + t % n : hist + (t - 6 * n);
    if (restore) *p = buf[t];
    else buf[t] = *p;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) {
    if (restore) hst[threadIdx.x] = ibuf[threadIdx.x];
    else ibuf[threadIdx.x] = hst[threadIdx.x];
  }
}

}  // namespace

namespace rx {
void snapshot(const Launch& L, Sys s, double* hist, int nhist_doubles, int* hst, double* buf, int* ibuf, int restore) {
  k_snapshot<<<4 * 152, 256, 0, L.st>>>(s, hist, nhist_doubles, hst, buf, ibuf, restore);
  *L.count += 1;
}
template <typename R> void chain_rule(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc) {
  // two threads per atom: about one pass over the canonical bonds of molecular systems (the
  // loops stride over any more)
  const unsigned grid = grid_for(2LL * s.n, 128);
  k_chain1<<<grid, 128, 0, L.st>>>(s, b, a);
  k_chain2<R><<<grid, 128, 0, L.st>>>(s, b, a, acc);
  *L.count += 2;
}
template void chain_rule<double>(const Launch&, Sys, BondList, AtomQ, Accum);
template void chain_rule<float>(const Launch&, Sys, BondList, AtomQ, Accum);

void finalize_forces(const Launch& L, Sys s, double* F) {
  k_finalize<<<grid_for(s.n, 256), 256, 0, L.st>>>(s, F);
  *L.count += 1;
}
void reduce_energies(const Launch& L, Sys s, Accum acc, const double* mass_t, const RedPlan& rp, double* E_rep,
                     double* vir_rep, double* ke_rep, double* etot, int* etot_idx) {
  k_reduce<<<dim3(rp.nchunk, NQ_RED), RED_BLOCK, 0, L.st>>>(s, acc, mass_t, rp, E_rep, vir_rep, ke_rep, etot, etot_idx);
  *L.count += 1;
}
void verlet_kick_drift(const Launch& L, Sys s, const double* mass_t, double dt, int drift, const CandList* cl) {
  k_kick_drift<<<grid_for(s.n, 256), 256, 0, L.st>>>(s, mass_t, dt, drift, cl ? 1 : 0, cl ? cl->half_skin2 : 0.0);
  *L.count += 1;
}

}  // namespace rx

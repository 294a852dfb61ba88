// (d) Tapered, shielded van der Waals and Coulomb terms, and the polarisation energy.
//
// Paper: Sec. 3.3 "Pairwise Interactions" and Algorithm 2 (threaded non-bonded loop:
// vdW + Coulomb per neighbour pair, energy reduction, private force arrays). GPU form:
// one warp per atom over its full far-list row (owner computes: each direction of a pair
// is evaluated by its own atom, so the atom's force needs no atomics and no
// thread-private copies; the energy and virial take half of each direction).
//
//   E_vdW  = Tap(r) D [e^{a (1 - f13/rv)} - 2 e^{a/2 (1 - f13/rv)}],
//            f13 = (r^p_vdW1 + gw^-p_vdW1)^(1/p_vdW1)
//   E_coul = Tap(r) k_e q_i q_j / (r^3 + gamma^-3)^(1/3)
//   E_pol  = chi_i q_i + eta_i q_i^2 / 2
//   Tap(x) = 20x^7 - 70x^6 + 84x^5 - 35x^4 + 1, x = r / r_nb
#include "reax_internal.cuh"

namespace {

inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }

template <typename R> struct QLoad;
template <> struct QLoad<double> {
  static __device__ __forceinline__ double get(const Sys& s, int j) { return s.q[j]; }
};
template <> struct QLoad<float> {
  static __device__ __forceinline__ float get(const Sys& s, int j) { return s.qf[j]; }
};

// one directed pair: accumulates energies, force on i and half the pair virial.
// FAST selects the MUFU-based pow/exp (used for pairs beyond r_bond in FP32).
template <typename R, bool FAST, typename A>
__device__ __forceinline__ void nb_pair(const Sys& s, const DParams<R>* __restrict__ P, int i, int j, int code, int r,
                                        int ti, R qi, R wv, R wc, A& ev, A& ec, A& fx, A& fy, A& fz, A* w) {
  R dx, dy, dz, qj;
  int tj;
  if constexpr (sizeof(R) == 4) {
    float4 hj, lj;
    PairVec<float>::getv(s, i, j, code, r, dx, dy, dz, hj, lj);   // charge and type ride along
    qj = hj.w;
    tj = rec_type(lj.w);
  } else {
    PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
    qj = QLoad<R>::get(s, j);
    tj = s.type[j];
  }
  const R r2 = dx * dx + dy * dy + dz * dz;
  const R rr = m_sqrt(r2);
  R tap, dtap;
  taper<R>(rr, P->r_nb, tap, dtap);
  const int pt = ti * MAXT + tj;
  const R pv = P->p_vdW1, ipv = R(1) / P->p_vdW1;
  // van der Waals
  const R rp = FAST ? f_pow(rr, pv) : m_pow(rr, pv);
  const R base = rp + P->vdw_gw_pow[pt];
  const R f13 = FAST ? f_pow(base, ipv) : m_pow(base, ipv);
  const R df13 = f13 * rp / (rr * base);
  const R al = P->vdw_alpha[pt], rv = P->vdw_rv[pt], D = P->vdw_D[pt];
  const R xr = R(1) - f13 / rv;
  const R E1 = FAST ? f_exp(al * xr) : m_exp(al * xr);
  const R E2 = FAST ? f_exp(R(0.5) * al * xr) : m_exp(R(0.5) * al * xr);
  const R evp = D * (E1 - R(2) * E2);
  const R devp = -(D * al / rv) * (E1 - E2);
  // Coulomb
  const R sh3 = r2 * rr + P->gamma_m3[pt];
  const R ish = FAST ? f_pow(sh3, R(-1) / R(3)) : R(1) / m_cbrt(sh3);
  const R kq = P->k_e * qi * qj;
  const R ecp = kq * ish;
  const R decp = -kq * r2 * ish * ish * ish * ish;
  ev += (A)(tap * evp);
  ec += (A)(tap * ecp);
  const R de = wv * (dtap * evp + tap * devp * df13) + wc * (dtap * ecp + tap * decp);
  const R c = de / rr;                                // F_i += (dE/dr) d/r
  fx += (A)(c * dx);
  fy += (A)(c * dy);
  fz += (A)(c * dz);
  // half of W_ab = -dE/dr d_a d_b / r for this direction
  const R hc = R(-0.5) * c;
  w[0] += (A)(hc * dx * dx); w[1] += (A)(hc * dy * dy); w[2] += (A)(hc * dz * dz);
  w[3] += (A)(hc * dx * dy); w[4] += (A)(hc * dx * dz); w[5] += (A)(hc * dy * dz);
}

// MUFU approximations (PTX ex2/lg2/rcp/rsqrt .approx): the far pairs' transcendentals run
// at these accuracies already (pow and exp as ex2(y lg2 x)), and they replace the
// correctly rounded square root and divisions there as well
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqa(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// one far directed pair (r_bond <= r < r_nb) on the mixed path: the terms of nb_pair with
// r^-1 from rsqrt, x^y = 2^(y log2 x), e^x = 2^(x log2 e) and reciprocals by rcp. The image
// vector is the plain FP32 difference of the hi parts plus that of the lo parts: its error
// (half an ulp of the hi difference, < 4e-6 A for a 100 A box) is < 1e-6 of r at r >= r_bond,
// far below the accuracy of these approximations. Atom i's records, the box halves, the
// constants of the pair type (`pt`: 2 x float4, see DParams::nbf) and the image signs
// (`sg`, one float4 per code) come from the caller. Accumulates the force and the UNSCALED
// pair virial d F^T (the caller multiplies by -1/2).
struct FarAtom {
  float4 hi, li;
  float Lhx, Lhy, Lhz, Llx, Lly, Llz;
  float kqi, wv, wc, iRc, pv, ipv;
};
template <typename A>
__device__ __forceinline__ void nb_pair_far(const Sys& s, const FarAtom& a, const float4* __restrict__ sg_tab,
                                            const float4* __restrict__ pt_tab, int j, int code, A& ev, A& ec,
                                            A& fx, A& fy, A& fz, A* w) {
  const float4 hj = s.ph[j], lj = s.pl[j];
  const float4 sg = sg_tab[code];
  const float dx = fmaf(sg.x, a.Lhx, hj.x - a.hi.x) + fmaf(sg.x, a.Llx, lj.x - a.li.x);
  const float dy = fmaf(sg.y, a.Lhy, hj.y - a.hi.y) + fmaf(sg.y, a.Lly, lj.y - a.li.y);
  const float dz = fmaf(sg.z, a.Lhz, hj.z - a.hi.z) + fmaf(sg.z, a.Llz, lj.z - a.li.z);
  const float r2 = dx * dx + dy * dy + dz * dz;
  const float ir = rsqa(r2);
  const float rr = r2 * ir;
  const float x = rr * a.iRc, x2 = x * x, x3 = x2 * x;
  const float tap = ((((20.0f * x - 70.0f) * x + 84.0f) * x - 35.0f) * x2 * x2) + 1.0f;
  const float dtap = ((((140.0f * x - 420.0f) * x + 420.0f) * x - 140.0f) * x3) * a.iRc;
  const float4 c0 = pt_tab[2 * rec_type(lj.w)], c1 = pt_tab[2 * rec_type(lj.w) + 1];
  // van der Waals
  const float rp = ex2a(a.pv * lg2a(rr));
  const float base = rp + c0.x;
  const float f13 = ex2a(a.ipv * lg2a(base));
  const float df13 = f13 * rp * ir * rcpa(base);
  const float t = c0.y * fmaf(-f13, c0.z, 1.0f);          // alpha (1 - f13/rv) log2(e)
  const float E1 = ex2a(t), E2 = ex2a(0.5f * t);
  const float evp = c0.w * fmaf(-2.0f, E2, E1);
  const float devp = c1.y * (E1 - E2);
  // Coulomb
  const float sh3 = fmaf(r2, rr, c1.x);
  const float ish = ex2a(-0.333333343f * lg2a(sh3));
  const float kq = a.kqi * hj.w;
  const float ecp = kq * ish;
  const float ish2 = ish * ish;
  const float decp = -kq * r2 * ish2 * ish2;
  ev += (A)(tap * evp);
  ec += (A)(tap * ecp);
  const float de = a.wv * (dtap * evp + tap * devp * df13) + a.wc * (dtap * ecp + tap * decp);
  const float c = de * ir;
  const float px = c * dx, py = c * dy, pz = c * dz;
  fx += (A)px;
  fy += (A)py;
  fz += (A)pz;
  w[0] += (A)(px * dx); w[1] += (A)(py * dy); w[2] += (A)(pz * dz);
  w[3] += (A)(px * dy); w[4] += (A)(px * dz); w[5] += (A)(py * dz);
}

template <typename R>
__device__ __forceinline__ void nonbonded_atom(const Sys& s, const FarList& f, const Accum& acc,
                                               const DParams<R>* __restrict__ P, unsigned mask) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  // mixed path: image signs per shift code and the far-pair constants, staged once per block
  __shared__ float4 sg_tab[27];
  __shared__ float4 pt_tab[MAXT * MAXT * 2];
  if constexpr (sizeof(R) == 4) {
    for (int t = threadIdx.x; t < 27 + MAXT * MAXT * 2; t += blockDim.x) {
      if (t < 27) {
        sg_tab[t] = make_float4((float)(t / 9 - 1), (float)((t / 3) % 3 - 1), (float)(t % 3 - 1), 0.0f);
      } else {
        const float* c = reinterpret_cast<const float*>(P->nbf) + 4 * (t - 27);
        pt_tab[t - 27] = make_float4(c[0], c[1], c[2], c[3]);
      }
    }
    __syncthreads();
  }
  if (i >= s.n) return;
  const int ti = s.type[i];
  const int r = s.rep[i];
  const R qi = QLoad<R>::get(s, i);
  const R wv = ((mask >> T_VDW) & 1u) ? R(1) : R(0);
  const R wc = ((mask >> T_COUL) & 1u) ? R(1) : R(0);
  // near part (r < r_bond): accurate math; per-lane sums in the path precision kept apart
  // from the far part (the near forces are ~100x larger; mixing would round the far ones away)
  R nev = 0, nec = 0, nfx = 0, nfy = 0, nfz = 0, nw[6] = {0, 0, 0, 0, 0, 0};
  const int nn = f.cntn[i], rown = i * f.capn;
  for (int k = lane; k < nn; k += 32)
    nb_pair<R, false, R>(s, P, i, f.jn[rown + k], f.sn[rown + k], r, ti, qi, wv, wc, nev, nec, nfx, nfy, nfz, nw);
  // far part (r_bond <= r < r_nb): MUFU pow/exp in FP32
  R lev = 0, lec = 0, lfx = 0, lfy = 0, lfz = 0, lw[6] = {0, 0, 0, 0, 0, 0};
  const int nfa = f.cnt[i], rowf = i * f.cap;
  if constexpr (sizeof(R) == 4) {
    FarAtom a;
    a.hi = s.ph[i];
    a.li = s.pl[i];
    a.Lhx = s.boxh[3 * r]; a.Lhy = s.boxh[3 * r + 1]; a.Lhz = s.boxh[3 * r + 2];
    a.Llx = s.boxl[3 * r]; a.Lly = s.boxl[3 * r + 1]; a.Llz = s.boxl[3 * r + 2];
    a.kqi = P->k_e * qi;
    a.wv = wv; a.wc = wc;
    a.iRc = 1.0f / P->r_nb; a.pv = P->p_vdW1; a.ipv = 1.0f / P->p_vdW1;
    const float4* pt = pt_tab + 2 * MAXT * ti;
    for (int k = lane; k < nfa; k += 32)
      nb_pair_far<R>(s, a, sg_tab, pt, f.j[rowf + k], f.s[rowf + k], lev, lec, lfx, lfy, lfz, lw);
#pragma unroll
    for (int q = 0; q < 6; ++q) lw[q] *= -0.5f;        // half of W_ab = -dE/dr d_a d_b / r (exact)
  } else {
    for (int k = lane; k < nfa; k += 32)
      nb_pair<R, true, R>(s, P, i, f.j[rowf + k], f.s[rowf + k], r, ti, qi, wv, wc, lev, lec, lfx, lfy, lfz, lw);
  }
  if constexpr (sizeof(R) == 4) {
    // near + far partials joined error-free per lane, float-float warp totals (FP32 only),
    // then lane q handles value q: the FP64 conversions are one warp instruction each
    constexpr int NVN = 11;   // 0-2 F_i; 3 E_vdW; 4 E_Coulomb; 5-10 virial
    const float nv[NVN] = {nfx, nfy, nfz, nev, nec, nw[0], nw[1], nw[2], nw[3], nw[4], nw[5]};
    const float fv[NVN] = {lfx, lfy, lfz, lev, lec, lw[0], lw[1], lw[2], lw[3], lw[4], lw[5]};
    float hi[NVN], lo[NVN];
#pragma unroll
    for (int q = 0; q < NVN; ++q) {
      two_sum(nv[q], fv[q], hi[q], lo[q]);
      warp_sum_ff2(hi[q], lo[q]);
    }
    float h, l;
    lane_pick<NVN>(hi, lo, lane, h, l);
    // fixed-point accumulators through 32-bit conversions (no FP64 instruction per value)
    if (lane < 3) {
      fix_add_ff((lane == 0 ? s.fx : lane == 1 ? s.fy : s.fz) + i, h, l, s.err);
    } else if (lane < 5) {
      fix_add_ff(acc.efx + (size_t)(T_VDW + lane - 3) * s.n + i, 0.5f * h, 0.5f * l, s.err);   // exact halving
    } else if (lane < NVN) {
      fix_add_ff(acc.vfx + (size_t)(lane - 5) * s.n + i, h, l, s.err);
    } else if (lane == NVN) {
      const double q = s.q[i];
      acc.e[T_POL * s.n + i] = (double)P->chi[ti] * q + 0.5 * (double)P->eta[ti] * q * q;
    }
  } else {
    const double ev = warp_sum_d(nev) + warp_sum_d(lev), ec = warp_sum_d(nec) + warp_sum_d(lec);
    const double fx = warp_sum_d(nfx) + warp_sum_d(lfx), fy = warp_sum_d(nfy) + warp_sum_d(lfy);
    const double fz = warp_sum_d(nfz) + warp_sum_d(lfz);
    double w[6];
    for (int q = 0; q < 6; ++q) w[q] = warp_sum_d(nw[q]) + warp_sum_d(lw[q]);
    if (lane == 0) {
      acc.e[T_VDW * s.n + i] = 0.5 * ev;
      acc.e[T_COUL * s.n + i] = 0.5 * ec;
      const double q = s.q[i];
      acc.e[T_POL * s.n + i] = (double)P->chi[ti] * q + 0.5 * (double)P->eta[ti] * q * q;
      fix_add(s.fx + i, fx, s.err);
      fix_add(s.fy + i, fy, s.err);
      fix_add(s.fz + i, fz, s.err);
      for (int q6 = 0; q6 < 6; ++q6) acc.vir[q6 * s.n + i] += w[q6];
    }
  }
}

// the FP32 form capped at 64 registers (72 uncapped; 12 bytes of spills): 32 warps per SM
// instead of 28 for this latency-bound kernel (petn32k 0.152 -> 0.147 ms); the FP64 form
// keeps its 126 registers
__global__ void __maxnreg__(64) k_nonbonded_f(Sys s, FarList f, Accum acc, const DParams<float>* __restrict__ P,
                                             unsigned mask) {
  nonbonded_atom<float>(s, f, acc, P, mask);
}
__global__ void k_nonbonded_d(Sys s, FarList f, Accum acc, const DParams<double>* __restrict__ P, unsigned mask) {
  nonbonded_atom<double>(s, f, acc, P, mask);
}

}  // namespace

namespace rx {
template <typename R>
void nonbonded(const Launch& L, Sys s, FarList f, Accum acc, const DParams<R>* P, unsigned mask) {
  const int bs = L.t().nb_block;
  if constexpr (sizeof(R) == 4) k_nonbonded_f<<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, f, acc, P, mask);
  else k_nonbonded_d<<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, f, acc, P, mask);
  *L.count += 1;
}
template void nonbonded<double>(const Launch&, Sys, FarList, Accum, const DParams<double>*, unsigned);
template void nonbonded<float>(const Launch&, Sys, FarList, Accum, const DParams<float>*, unsigned);
}  // namespace rx

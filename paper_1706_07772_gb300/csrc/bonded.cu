// (b) bond-order correction and (c) bonded terms, with their dE/dBO and dE/dDelta parts.
//
// Paper: Sec. 2.1 (bond orders, lone pair, over/under-coordination, valence angle,
// torsion, conjugation, H-bond), Sec. 3.3 "Pairwise Interactions" (bond-order correction,
// bond energy), "Three-body Interactions" (angles identified per central atom) and the
// 4-body terms built on top of the bonds (Table 2 "Bond Orders", "3-body", "4-body").
//
// GPU form: every per-interaction derivative is split into (1) a geometric part,
// applied at once as forces (and virial) through dE/d(interaction vectors), and (2)
// dE/dBO, dE/dBO_pi, dE/dBO_pipi per bond entry and dE/d(sum BO) per atom, accumulated
// in int64 fixed point and turned into forces by the chain-rule pass (forces.cu).
// Warp per central atom (angles, H-bonds) or per central bond (torsions): lanes
// enumerate the pairs of the centre's bonds, so skewed per-atom work stays inside one
// warp's loop instead of one thread's.
//
// Functional forms (energy kcal/mol; symbols as in the parameter tables):
//  BO correction  f1 = (A_i + A_j)/2, A_x = (V_x + f2)/(V_x + f2 + f3),
//                 f2 = e^{-p_boc1 D'_i} + e^{-p_boc1 D'_j},
//                 f3 = -(1/p_boc2) ln((e^{-p_boc2 D'_i} + e^{-p_boc2 D'_j})/2),
//                 f4 = 1/(1 + e^{-p_boc3 (p_boc4 BO'^2 - D'boc_i) + p_boc5}) (f5 with j),
//                 BO = BO' f1 f4 f5, BO_pi = BO'_pi f1^2 f4 f5, BO_pp = BO'_pp f1^2 f4 f5
//  bond           -De_s BOs e^{p_be1 (1 - BOs^p_be2)} - De_p BO_pi - De_pp BO_pp
//  lone pair      p_lp2 Dlp / (1 + e^{-75 Dlp}),  n_lp = e^{-p_lp1 (2 + De - 2T)^2} - T,
//                 T = trunc(De/2), Dlp = (Vale - Val)/2 - n_lp
//  over           (sum p_ovun1 De_s BO) Dlpc/(Dlpc + Val + 1e-8) / (1 + e^{p_ovun2 Dlpc})
//  under          -p_ovun5 (1 - e^{p_ovun6 Dlpc}) / (1 + e^{-p_ovun2 Dlpc})
//                 / (1 + p_ovun7 e^{p_ovun8 S}),  Dlpc = D - Dlp/(1 + p_ovun3 e^{p_ovun4 S}),
//                 S = sum_j (D_j - Dlp_j)(BO_pi + BO_pp)
//  valence        f7(BO_ij) f7(BO_jk) f8(Dang_j) p_val1 (1 - e^{-p_val2 (th0 - th)^2})
//  penalty        p_pen1 f9(D_j) e^{-p_pen2 (BO_ij - 2)^2} e^{-p_pen2 (BO_jk - 2)^2}
//  coalition      p_coa1/(1 + e^{p_coa2 Dang_j}) e^{-p_coa3 (SBO_i - BO_ij)^2}
//                 e^{-p_coa3 (SBO_k - BO_jk)^2} e^{-p_coa4 (BO_ij - 1.5)^2} e^{-p_coa4 (BO_jk - 1.5)^2}
//  torsion        f10 sin th1 sin th2 [V1 (1 + cos w)/2 + V2 e^{p_tor1 (2 - BO_pi,jk - f11)^2}
//                 (1 - cos 2w)/2 + V3 (1 + cos 3w)/2]
//  conjugation    p_cot1 prod e^{-p_cot2 (BO - 1.5)^2} [1 + (cos^2 w - 1) sin th1 sin th2]
//  H-bond         p_hb1 (1 - e^{-p_hb2 BO_XH}) e^{-p_hb3 (r0/r + r/r0 - 2)} sin^4(th/2)
#include "reax_internal.cuh"

namespace {

inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }

template <typename R> __device__ __forceinline__ R wbit(unsigned mask, int t) {
  return ((mask >> t) & 1u) ? R(1) : R(0);
}

// ------------------------------------------------------------------ BO correction
// Evaluated in the path's precision R from FP64 Delta' and BO'; the factors and their
// partials are stored in FP64 for the chain rule, BO, BO_pi and BO_pp in R. One thread per
// unordered bond writes both directed entries: the canonical entry e of atom i and its
// mirror m in atom j's row. f1, F = f1 f4 f5 and G = f1^2 f4 f5 are symmetric; f4/f5 (stored
// as the entry's own factor fo and the other atom's ft), their BO' derivatives and the
// Delta' derivatives df1, dfo_d belong to one atom each, so the mirror holds them with the
// roles swapped. Every value comes from the same operands, in the same order, as an
// evaluation of that entry alone.
template <typename R>
__global__ void k_bo_correct(Sys s, BondList bl, AtomQ aq, const DParams<R>* __restrict__ P) {
  const int nc = *bl.ncanon;
  const double* BOp = bl.bop;
  const double* BOpi = bl.bopi;
  const double* BOpp = bl.bopp;
  R* bo = (R*)bl.bo; R* bo_pi = (R*)bl.bo_pi; R* bo_pp = (R*)bl.bo_pp;
  double* f1a = (double*)bl.f1; double* foa = (double*)bl.fo; double* fta = (double*)bl.ft;
  double* df1a = (double*)bl.df1; double* dfoba = (double*)bl.dfo_bo; double* dftba = (double*)bl.dft_bo;
  double* dfoda = (double*)bl.dfo_d;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
    const int e = bl.canon[t];
    const int i = e / bl.cap;
    const int j = bl.j[e];
    const int m = bl.mirror[e];
    const int ti = s.type[i], tj = s.type[j];
    const int pt = ti * MAXT + tj;
    const R bp = (R)BOp[e];
    R f1 = 1, df1i = 0, df1j = 0;
    if (P->ovc[pt] > R(0)) {
      // i is the lower atom of the bond (canonical entry)
      const R dlo = (R)aq.dp[i], dhi = (R)aq.dp[j];
      const R vlo = P->val[ti], vhi = P->val[tj];
      const R e1lo = m_expc(-P->p_boc1 * dlo), e1hi = m_expc(-P->p_boc1 * dhi);
      const R f2 = e1lo + e1hi;
      // f3 = -(1/p_boc2) ln((e^a + e^b)/2), a,b = -p_boc2 D'; as a log-sum-exp so that
      // neither underflow (both exponentials 0) nor overflow reaches the log or df3
      const R ga = -P->p_boc2 * dlo, gb = -P->p_boc2 * dhi;
      const R gm = ga > gb ? ga : gb;
      const R wlo = m_exp(ga - gm), whi = m_exp(gb - gm);
      const R wsum = wlo + whi;
      const R f3 = -(R(1) / P->p_boc2) * (gm + m_log(R(0.5) * wsum));
      const R dlo_den = vlo + f2 + f3, dhi_den = vhi + f2 + f3;
      f1 = R(0.5) * ((vlo + f2) / dlo_den + (vhi + f2) / dhi_den);
      // df1/dDelta'_i (entry e) and df1/dDelta'_j (entry m)
      {
        const R df2 = -P->p_boc1 * e1lo;
        const R df3 = wlo / wsum;
        const R dAlo = (f3 * df2 - (vlo + f2) * df3) / (dlo_den * dlo_den);
        const R dAhi = (f3 * df2 - (vhi + f2) * df3) / (dhi_den * dhi_den);
        df1i = R(0.5) * (dAlo + dAhi);
      }
      {
        const R df2 = -P->p_boc1 * e1hi;
        const R df3 = whi / wsum;
        const R dAlo = (f3 * df2 - (vlo + f2) * df3) / (dlo_den * dlo_den);
        const R dAhi = (f3 * df2 - (vhi + f2) * df3) / (dhi_den * dhi_den);
        df1j = R(0.5) * (dAlo + dAhi);
      }
    }
    // f4 (atom i) and f5 (atom j), their BO' and Delta'boc derivatives
    R fi = 1, fj = 1, dfi_bo = 0, dfj_bo = 0, dfi_d = 0, dfj_d = 0;
    if (P->v13[pt] > R(0)) {
      const R p3 = P->p_boc3[pt], p4 = P->p_boc4[pt], p5 = P->p_boc5[pt];
      R sdi, sdj;
      sig_pair<R>(-p3 * (p4 * bp * bp - (R)aq.dpboc[i]) + p5, fi, sdi);
      sig_pair<R>(-p3 * (p4 * bp * bp - (R)aq.dpboc[j]) + p5, fj, sdj);
      dfi_bo = R(2) * p3 * p4 * bp * sdi;
      dfj_bo = R(2) * p3 * p4 * bp * sdj;
      dfi_d = -p3 * sdi;
      dfj_d = -p3 * sdj;
    }
    const double flo = fi, fhi = fj;
    const double F = (double)f1 * flo * fhi;
    const double G = (double)f1 * f1 * flo * fhi;
    const R b = (R)(BOp[e] * F), bpi = (R)(BOpi[e] * G), bpp = (R)(BOpp[e] * G);
    bo[e] = b; bo_pi[e] = bpi; bo_pp[e] = bpp;
    bo[m] = b; bo_pi[m] = bpi; bo_pp[m] = bpp;
    f1a[e] = f1; foa[e] = fi; fta[e] = fj; df1a[e] = df1i;
    dfoba[e] = dfi_bo; dftba[e] = dfj_bo; dfoda[e] = dfi_d;
    f1a[m] = f1; foa[m] = fj; fta[m] = fi; df1a[m] = df1j;
    dfoba[m] = dfj_bo; dftba[m] = dfi_bo; dfoda[m] = dfj_d;
  }
}

// ------------------------------------------------------------------ atom terms + lone pair
template <typename R>
__global__ void k_atom_terms(Sys s, BondList bl, AtomQ aq, Accum acc, const DParams<R>* __restrict__ P,
                             unsigned mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int ti = s.type[i];
  const int nb = bl.cnt[i];
  const R* bo = (const R*)bl.bo;
  const R* bo_pi = (const R*)bl.bo_pi;
  const R* bo_pp = (const R*)bl.bo_pp;
  double sumbo = 0, pisum = 0, sum8 = 0;                 // sums in FP64
  for (int k = 0; k < nb; ++k) {
    const int e = i * bl.cap + k;
    const R b = bo[e];
    const R b2 = b * b, b4 = b2 * b2;
    sumbo += (double)b;
    pisum += (double)(bo_pi[e] + bo_pp[e]);
    sum8 += (double)(b4 * b4);
  }
  const double delta = sumbo - (double)P->val[ti];
  const double dele = sumbo - (double)P->vale[ti];
  const double dang = sumbo - (double)P->valang[ti];
  const double T = trunc(dele * 0.5);
  const R el = (R)(2.0 + dele - 2.0 * T);
  const R enlp = m_exp(-P->p_lp1 * el * el);
  const double nlp = (double)enlp - T;
  const R dnlp = R(-2) * P->p_lp1 * el * enlp;
  const double dlp = 0.5 * ((double)P->vale[ti] - (double)P->val[ti]) - nlp;
  R sg, sgd;
  sig_pair<R>(R(-75) * (R)dlp, sg, sgd);                  // 1/(1+e^{-75 dlp})
  const R elp = P->p_lp2[ti] * (R)dlp * sg;
  const R delp = P->p_lp2[ti] * (sg + R(75) * (R)dlp * sgd);
  fix_add(aq.cddelta + i, wbit<R>(mask, T_LP) * delp * (-dnlp), s.err);
  const R prodexp = m_exp(-(R)sum8);
  const double sbo_fac = -dang - (double)P->p_val8 * nlp;
  const R sbo = (R)(pisum + (1.0 - (double)prodexp) * sbo_fac);
  R sbo2, dsbo2;
  const R p9 = P->p_val9;
  if (sbo <= R(0)) {
    sbo2 = 0; dsbo2 = 0;
  } else if (sbo < R(1)) {
    sbo2 = m_pow(sbo, p9);
    dsbo2 = p9 * m_pow(sbo, p9 - R(1));
  } else if (sbo < R(2)) {
    sbo2 = R(2) - m_pow(R(2) - sbo, p9);
    dsbo2 = p9 * m_pow(R(2) - sbo, p9 - R(1));
  } else {
    sbo2 = 2; dsbo2 = 0;
  }
  aq.sumbo[i] = sumbo;
  aq.delta[i] = delta;
  aq.dang[i] = dang;
  aq.sumbo_f[i] = (float)sumbo;
  aq.dang_f[i] = (float)dang;
  aq.nlp[i] = nlp;
  aq.dnlp[i] = dnlp;
  aq.dlp[i] = dlp;
  aq.dd[i] = delta - dlp;
  aq.prodexp[i] = prodexp;
  aq.sbo2[i] = sbo2;
  aq.dsbo2[i] = dsbo2;
  aq.sbo_fac[i] = sbo_fac;
  aq.delta_f[i] = (float)delta;
  aq.sbo2_f[i] = (float)sbo2;
  aq.dsbo2_f[i] = (float)dsbo2;
  aq.prodexp_f[i] = (float)prodexp;
  aq.sbo_fac_f[i] = (float)sbo_fac;
  aq.dnlp_f[i] = (float)dnlp;
  acc.e[T_LP * s.n + i] = elp;
}

// ------------------------------------------------------------------ over/under + bond energy
template <typename R>
__global__ void k_over_under_bond(Sys s, BondList bl, AtomQ aq, Accum acc, const DParams<R>* __restrict__ P,
                                  unsigned mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int ti = s.type[i];
  const int nb = bl.cnt[i];
  const R* bo = (const R*)bl.bo;
  const R* bo_pi = (const R*)bl.bo_pi;
  const R* bo_pp = (const R*)bl.bo_pp;
  double S = 0, sov = 0;
  for (int k = 0; k < nb; ++k) {
    const int e = i * bl.cap + k;
    const int j = bl.j[e];
    const int pt = ti * MAXT + s.type[j];
    S += aq.dd[j] * (double)(bo_pi[e] + bo_pp[e]);
    sov += (double)(P->p_ovun1[pt] * P->De_s[pt] * bo[e]);
  }
  const double delta = aq.delta[i], dlp = aq.dlp[i];
  const R dnlp = (R)aq.dnlp[i];
  const R V = P->val[ti];
  const R e4 = m_expc(P->p_ovun4 * (R)S);
  const R den = R(1) + P->p_ovun3 * e4;
  const R dlpc = (R)(delta - dlp / (double)den);
  const R ddlpc_dS = (R)dlp * P->p_ovun3 * P->p_ovun4 * e4 / (den * den);
  // over
  const R gd = dlpc + V + R(1e-8);
  const R g = dlpc / gd;
  const R dg = (V + R(1e-8)) / (gd * gd);
  const R p2 = P->p_ovun2[ti];
  R s1, s1d;
  sig_pair<R>(p2 * dlpc, s1, s1d);                     // 1/(1+e^{p2 dlpc})
  const R ds1 = -p2 * s1d;
  const R eover = (R)sov * g * s1;
  const R deover = (R)sov * (dg * s1 + g * ds1);
  // under
  const R em6 = m_expm1(P->p_ovun6 * dlpc);            // e^{p6 dlpc} - 1
  const R e6 = em6 + R(1);
  R s2, s2d;
  sig_pair<R>(-p2 * dlpc, s2, s2d);                    // 1/(1+e^{-p2 dlpc})
  const R ds2 = p2 * s2d;
  const R e8 = m_expc(P->p_ovun8 * (R)S);
  const R h = R(1) / (R(1) + P->p_ovun7 * e8);
  const R dh = -h * h * P->p_ovun7 * P->p_ovun8 * e8;
  const R p5 = P->p_ovun5[ti];
  const R eunder = p5 * em6 * s2 * h;
  const R deunder = -p5 * (-P->p_ovun6 * e6 * s2 + (-em6) * ds2) * h;
  const R deunder_S = p5 * em6 * s2 * dh;
  const R wo = wbit<R>(mask, T_OVER), wu = wbit<R>(mask, T_UNDER);
  const R cdlpc = wo * deover + wu * deunder;
  const R cds = cdlpc * ddlpc_dS + wu * deunder_S;
  fix_add(aq.cddelta + i, cdlpc * (R(1) + dnlp / den), s.err);
  aq.cds[i] = cds;
  acc.e[T_OVER * s.n + i] = eover;
  acc.e[T_UNDER * s.n + i] = eunder;
  const R dov_dsum = wo * g * s1;
  // bond energy on the canonical half of i's row
  const R wb = wbit<R>(mask, T_BOND);
  double ebond = 0.0;
  for (int k = 0; k < nb; ++k) {
    const int e = i * bl.cap + k;
    const int j = bl.j[e];
    const int pt = ti * MAXT + s.type[j];
    const R cdd = (R)aq.dd[j];
    R cb = dov_dsum * P->p_ovun1[pt] * P->De_s[pt];
    R cpi = cds * cdd, cpp = cds * cdd;
    if ((i < j) || (i == j && bl.s[e] > 13)) {
      const R b = bo[e], bpi = bo_pi[e], bpp = bo_pp[e];
      const R bs = b - bpi - bpp;
      R es = 0, des = 0;
      if (bs > R(0)) {
        const R pw = m_pow(bs, P->p_be2[pt]);
        const R ex = m_exp(P->p_be1[pt] * (R(1) - pw));
        es = -P->De_s[pt] * bs * ex;
        des = -P->De_s[pt] * ex * (R(1) - P->p_be1[pt] * P->p_be2[pt] * pw);
      }
      ebond += (double)(es - P->De_p[pt] * bpi - P->De_pp[pt] * bpp);
      cb += wb * des;
      cpi += wb * (-des - P->De_p[pt]);
      cpp += wb * (-des - P->De_pp[pt]);
    }
    fix_add(bl.cdbo + e, cb, s.err);
    fix_add(bl.cdbopi + e, cpi, s.err);
    fix_add(bl.cdbopp + e, cpp, s.err);
  }
  acc.e[T_BOND * s.n + i] = ebond;
}

// dE/dS_i reaches neighbour j through D_j - Dlp_j: gathered by j over its own row
template <typename R>
__global__ void k_s_gather(Sys s, BondList bl, AtomQ aq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int nb = bl.cnt[i];
  const R* bo_pi = (const R*)bl.bo_pi;
  const R* bo_pp = (const R*)bl.bo_pp;
  double acc = 0.0;
  for (int k = 0; k < nb; ++k) {
    const int e = i * bl.cap + k;
    acc += aq.cds[bl.j[e]] * (double)(bo_pi[e] + bo_pp[e]);
  }
  fix_add(aq.cddelta + i, acc * (1.0 + aq.dnlp[i]), s.err);
}

// ------------------------------------------------------------------ geometry helpers
template <typename R> struct Vec3 { R x, y, z; };
template <typename R> __device__ __forceinline__ R dot3(const Vec3<R>& a, const Vec3<R>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R> __device__ __forceinline__ Vec3<R> lin2(R a, const Vec3<R>& u, R b, const Vec3<R>& v) {
  return Vec3<R>{a * u.x + b * v.x, a * u.y + b * v.y, a * u.z + b * v.z};
}
template <typename R> __device__ __forceinline__ Vec3<R> cross3(const Vec3<R>& a, const Vec3<R>& b) {
  return Vec3<R>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// cross product with each component a correctly-rounded difference of products
template <typename R> __device__ __forceinline__ Vec3<R> cross_acc(const Vec3<R>& a, const Vec3<R>& b) {
  return Vec3<R>{diff_prod(a.y, b.z, a.z, b.y), diff_prod(a.z, b.x, a.x, b.z), diff_prod(a.x, b.y, a.y, b.x)};
}
template <typename R>
__device__ __forceinline__ Vec3<R> load_vec(const BondList& bl, int e) {
  return Vec3<R>{((const R*)bl.dx)[e], ((const R*)bl.dy)[e], ((const R*)bl.dz)[e]};
}
template <typename R>
__device__ __forceinline__ void force_add(const Sys& s, int a, R fx, R fy, R fz) {
  fix_add(s.fx + a, fx, s.err);
  fix_add(s.fy + a, fy, s.err);
  fix_add(s.fz + a, fz, s.err);
}
// virial W_ab -= g_a v_b (xx yy zz xy xz yz), per-lane partial in the path precision
template <typename R>
__device__ __forceinline__ void vir_sub(R* w, const Vec3<R>& g, const Vec3<R>& v) {
  w[0] -= g.x * v.x; w[1] -= g.y * v.y; w[2] -= g.z * v.z;
  w[3] -= g.x * v.y; w[4] -= g.x * v.z; w[5] -= g.y * v.z;
}
// f9-type function (2 + e^{-a D}) / (1 + e^{-a D} + e^{b D}) and its D-derivative,
// written with u = e^{-aD}/den, v = e^{bD}/den in [0, 1] so no intermediate overflows:
// df/dD = (a u - 2 b v)/den - (a + b) u v
template <typename R> __device__ __forceinline__ void f9fun(R a, R b, R D, R& f, R& df) {
  const R e3 = m_expc(-a * D), e4 = m_expc(b * D);
  const R den = R(1) + e3 + e4;
  const R u = e3 / den, v = e4 / den;
  f = R(2) / den + u;
  df = (a * u - R(2) * b * v) / den - (a + b) * u * v;
}

// ------------------------------------------------------------------ valence angles
template <typename R>
__global__ void k_angles(Sys s, BondList bl, AtomQ aq, Accum acc, const DParams<R>* __restrict__ P,
                         unsigned mask) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= s.n) return;
  const int nb = bl.cnt[j];
  if (nb < 2) return;
  const int tj = s.type[j];
  const R* bo = (const R*)bl.bo;
  const R dang = (R)aq.dang[j], delta = (R)aq.delta[j];
  const R sbo2 = (R)aq.sbo2[j];
  const R wv = wbit<R>(mask, T_VAL), wp = wbit<R>(mask, T_PEN), wc = wbit<R>(mask, T_COA);
  // centre-only factors
  const R pv5 = P->p_val5[tj];
  const R e6 = m_expc(P->p_val6 * dang);
  const R ex2 = m_exp(-P->p_val10 * (R(2) - sbo2));
  const R dth0_dsbo2 = ex2 * P->p_val10;              // times th00
  R f9, df9;
  f9fun<R>(P->p_pen3, P->p_pen4, delta, f9, df9);
  R scoa, scoad;
  sig_pair<R>(P->p_coa2 * dang, scoa, scoad);
  R l_eval = 0, l_epen = 0, l_ecoa = 0, l_cdsbo = 0, l_cdd = 0;    // per-lane partials
  R l_fj[3] = {0, 0, 0}, l_w[6] = {0, 0, 0, 0, 0, 0};
  const int npair = nb * (nb - 1) / 2;
  for (int p = lane; p < npair; p += 32) {
    int a = 0, rem = p;
    while (rem >= nb - 1 - a) { rem -= nb - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const int ea = j * bl.cap + a, eb = j * bl.cap + b;
    const R BOa = bo[ea], BOb = bo[eb];
    if (!(BOa > P->thb_cut && BOb > P->thb_cut && BOa * BOb > P->thb_cutsq)) continue;
    const int i = bl.j[ea], k = bl.j[eb];
    const int ti = s.type[i], tk = s.type[k];
    const int t3 = (ti * MAXT + tj) * MAXT + tk;
    const Vec3<R> u = load_vec<R>(bl, ea), v = load_vec<R>(bl, eb);
    const R L1 = dot3(u, u), L2 = dot3(v, v);
    // theta = atan2(|u x v|, u.v): accurate at every angle; d theta/du = (u x n^)/|u|^2,
    // d theta/dv = (n^ x v)/|v|^2 with n^ = (u x v)/|u x v|
    const Vec3<R> nrm = cross_acc(u, v);
    const R nn = m_sqrt(dot3(nrm, nrm));
    const R th = m_atan2(nn, dot3(u, v));
    const bool cok = nn > R(0);
    // valence
    const R th00 = P->th00[t3];
    const R th0 = R(3.14159265358979323846) - th00 * (R(1) - ex2);
    const R pv3 = P->p_val3[tj], pv4 = P->p_val4[t3];
    const R pa = m_pow(BOa, pv4), pb = m_pow(BOb, pv4);
    const R ea7 = m_exp(-pv3 * pa), eb7 = m_exp(-pv3 * pb);
    const R f7a = -m_expm1(-pv3 * pa), f7b = -m_expm1(-pv3 * pb);
    const R df7a = ea7 * pv3 * pv4 * pa / BOa, df7b = eb7 * pv3 * pv4 * pb / BOb;
    // f8 = pv5 - (pv5 - 1)(2 + e6)/(1 + e6 + e7); with u = e6/den, v = e7/den:
    // d[(2 + e6)/den]/dDang = (2 p7 v - p6 u)/den + (p6 + p7) u v
    const R p7 = P->p_val7[t3];
    const R e7 = m_expc(-p7 * dang);
    const R den8 = R(1) + e6 + e7;
    const R u8 = e6 / den8, v8 = e7 / den8;
    const R f8 = pv5 - (pv5 - R(1)) * (R(2) / den8 + u8);
    const R df8 = -(pv5 - R(1)) * ((R(2) * p7 * v8 - P->p_val6 * u8) / den8 + (P->p_val6 + p7) * u8 * v8);
    const R pv1 = P->p_val1[t3], pv2 = P->p_val2[t3];
    const R D = th0 - th;
    const R exv = m_exp(-pv2 * D * D);
    const R gth = -m_expm1(-pv2 * D * D);
    const R Cv = f7a * f7b * f8 * pv1;
    const R ev = Cv * gth;
    const R dEdD = Cv * exv * R(2) * pv2 * D;          // d/dD of Cv (1 - e^{-pv2 D^2})
    const R dEv_dth = -dEdD;
    const R dEv_dsbo2 = dEdD * th00 * dth0_dsbo2;
    // penalty
    const R pp2 = P->p_pen2;
    const R ga = m_exp(-pp2 * (BOa - R(2)) * (BOa - R(2))), gb = m_exp(-pp2 * (BOb - R(2)) * (BOb - R(2)));
    const R ep = P->p_pen1[t3] * f9 * ga * gb;
    // coalition
    R sbi, sbk;
    if constexpr (sizeof(R) == 4) {
      sbi = aq.sumbo_f[i] - BOa;
      sbk = aq.sumbo_f[k] - BOb;
    } else {
      sbi = (R)(aq.sumbo[i] - (double)BOa);
      sbk = (R)(aq.sumbo[k] - (double)BOb);
    }
    const R pc3 = P->p_coa3, pc4 = P->p_coa4;
    const R ec = P->p_coa1[t3] * scoa * m_exp(-pc3 * sbi * sbi) * m_exp(-pc3 * sbk * sbk) *
                 m_exp(-pc4 * (BOa - R(1.5)) * (BOa - R(1.5))) * m_exp(-pc4 * (BOb - R(1.5)) * (BOb - R(1.5)));
    l_eval += ev;
    l_epen += ep;
    l_ecoa += ec;
    // bond-order and Delta derivatives
    const R dBOa = wv * df7a * f7b * f8 * pv1 * gth + wp * ep * (R(-2) * pp2 * (BOa - R(2))) +
                   wc * ec * (R(2) * pc3 * sbi - R(2) * pc4 * (BOa - R(1.5)));
    const R dBOb = wv * f7a * df7b * f8 * pv1 * gth + wp * ep * (R(-2) * pp2 * (BOb - R(2))) +
                   wc * ec * (R(2) * pc3 * sbk - R(2) * pc4 * (BOb - R(1.5)));
    fix_add(bl.cdbo + ea, dBOa, s.err);
    fix_add(bl.cdbo + eb, dBOb, s.err);
    fix_add(aq.cddelta + i, wc * ec * (R(-2) * pc3 * sbi), s.err);
    fix_add(aq.cddelta + k, wc * ec * (R(-2) * pc3 * sbk), s.err);
    l_cdd += wv * f7a * f7b * df8 * pv1 * gth + wp * P->p_pen1[t3] * df9 * ga * gb +
             wc * (scoa > R(0) ? -ec * P->p_coa2 * scoad / scoa : R(0));
    l_cdsbo += wv * dEv_dsbo2;
    // geometry: E depends on cos(theta) only through the valence term
    if (cok) {
      const R gt = wv * dEv_dth / nn;
      const Vec3<R> cu = cross3(u, nrm), cv = cross3(nrm, v);
      const Vec3<R> gu = Vec3<R>{gt * cu.x / L1, gt * cu.y / L1, gt * cu.z / L1};
      const Vec3<R> gv = Vec3<R>{gt * cv.x / L2, gt * cv.y / L2, gt * cv.z / L2};
      force_add<R>(s, i, -gu.x, -gu.y, -gu.z);
      force_add<R>(s, k, -gv.x, -gv.y, -gv.z);
      l_fj[0] += gu.x + gv.x; l_fj[1] += gu.y + gv.y; l_fj[2] += gu.z + gv.z;
      vir_sub(l_w, gu, u);
      vir_sub(l_w, gv, v);
    }
  }
  if constexpr (sizeof(R) == 4) {
    // float-float warp totals (FP32 only); then lane q handles value q, so each FP64
    // conversion or update below is one warp instruction for all values
    constexpr int NVA = 14;   // 0-2 E_val, E_pen, E_coa; 3-5 F_j; 6-11 virial; 12 dE/dSBO2; 13 dE/dDelta
    float hi[NVA] = {l_eval, l_epen, l_ecoa, l_fj[0], l_fj[1], l_fj[2], l_w[0], l_w[1], l_w[2], l_w[3], l_w[4],
                     l_w[5], l_cdsbo, l_cdd};
    float lo[NVA];
#pragma unroll
    for (int q = 0; q < NVA; ++q) {
      lo[q] = 0.0f;
      warp_sum_ff2(hi[q], lo[q]);
    }
    float h, l;
    lane_pick<NVA>(hi, lo, lane, h, l);
    const double d = (double)h + (double)l;
    const double cdsbo = ((double)hi[12] + (double)lo[12]) * aq.dsbo2[j];   // dE/dSBO
    const double prod = aq.prodexp[j];
    if (lane < 3) {
      acc.e[(T_VAL + lane) * s.n + j] = d;
    } else if (lane < 6) {
      fix_add_ff((lane == 3 ? s.fx : lane == 4 ? s.fy : s.fz) + j, h, l, s.err);
    } else if (lane < 12) {
      acc.vir[(lane - 6) * s.n + j] += d;
    } else if (lane == 13) {
      const double dsbo_dsum = -(1.0 - prod) * (1.0 + (double)P->p_val8 * aq.dnlp[j]);
      fix_add(aq.cddelta + j, d + cdsbo * dsbo_dsum, s.err);
    }
    // SBO depends on every bond of j: distribute dE/dSBO over j's row (FP32 terms)
    if (cdsbo != 0.0) {
      const float cf = (float)cdsbo, pf = (float)prod, ff = (float)aq.sbo_fac[j];
      for (int k = lane; k < nb; k += 32) {
        const int e = j * bl.cap + k;
        const float b = bo[e];
        const float b2 = b * b, b4 = b2 * b2;
        fix_add(bl.cdbopi + e, cf, s.err);
        fix_add(bl.cdbopp + e, cf, s.err);
        fix_add(bl.cdbo + e, cf * pf * 8.0f * b4 * b2 * b * ff, s.err);
      }
    }
  } else {
    const double eval = warp_sum_d(l_eval), epen = warp_sum_d(l_epen), ecoa = warp_sum_d(l_ecoa);
    double cdsbo = warp_sum_d(l_cdsbo);
    const double cdd = warp_sum_d(l_cdd);
    double fj[3], w[6];
    for (int q = 0; q < 3; ++q) fj[q] = warp_sum_d(l_fj[q]);
    for (int q = 0; q < 6; ++q) w[q] = warp_sum_d(l_w[q]);
    cdsbo *= aq.dsbo2[j];                                // dE/dSBO
    const double prod = aq.prodexp[j];
    if (lane == 0) {
      acc.e[T_VAL * s.n + j] = eval;
      acc.e[T_PEN * s.n + j] = epen;
      acc.e[T_COA * s.n + j] = ecoa;
      force_add<double>(s, j, fj[0], fj[1], fj[2]);
      const double dsbo_dsum = -(1.0 - prod) * (1.0 + (double)P->p_val8 * aq.dnlp[j]);
      fix_add(aq.cddelta + j, cdd + cdsbo * dsbo_dsum, s.err);
      for (int q = 0; q < 6; ++q) acc.vir[q * s.n + j] += w[q];
    }
    // SBO depends on every bond of j: distribute dE/dSBO over j's row
    if (cdsbo != 0.0) {
      const double fac = aq.sbo_fac[j];
      for (int k = lane; k < nb; k += 32) {
        const int e = j * bl.cap + k;
        const double b = (double)bo[e];
        const double b2 = b * b, b4 = b2 * b2;
        fix_add(bl.cdbopi + e, cdsbo, s.err);
        fix_add(bl.cdbopp + e, cdsbo, s.err);
        fix_add(bl.cdbo + e, cdsbo * prod * 8.0 * b4 * b2 * b * fac, s.err);
      }
    }
  }
}

// ------------------------------------------------------------------ torsion + conjugation
// One group of TG lanes per canonical bond j-k (the central bond; j < k, or the same atom
// through a periodic image with shift code > 13). The group's lanes take the
// (nb_j - 1)(nb_k - 1) choices of an outer bond i-j and l-k; per-quadruple terms go to i, l
// and the outer bonds by fixed-point atomics, the group totals for j, k and the central
// bond are combined inside the group (float-float on the mixed path) and added by fixed-
// point atomics, energies and virial into per-atom fixed-point accumulators. Integer
// atomics make the result independent of scheduling.

template <typename R, int TG> struct GroupSum;
template <int TG> struct GroupSum<float, TG> {
  // every lane of the TG-lane group gets the group total (hi, lo)
  static __device__ __forceinline__ void run(float& hi, float& lo) {
#pragma unroll
    for (int o = TG / 2; o > 0; o >>= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
      float s, e;
      two_sum(hi, ohi, s, e);
      lo = __fadd_rn(__fadd_rn(lo, olo), e);
      hi = s;
    }
  }
  static __device__ __forceinline__ void add(unsigned long long* p, float hi, float lo, int* err) {
    fix_add_ff(p, hi, lo, err);
  }
};
template <int TG> struct GroupSum<double, TG> {
  static __device__ __forceinline__ void run(double& hi, double& lo) {
#pragma unroll
    for (int o = TG / 2; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
    lo = 0.0;
  }
  static __device__ __forceinline__ void add(unsigned long long* p, double hi, double lo, int* err) {
    fix_add(p, hi + lo, err);
  }
};

// Mixed path with G lanes per centre atom (32 / G centres per warp): molecular centres have
// few bond pairs (about 9 at this density, half passing the thresholds), so a whole warp per
// centre would leave most lanes idle. The group's float-float totals come from group
// butterflies; lane q of the group then converts and stores totals q, q + G, ...
template <int G>
__global__ void __maxnreg__(72) k_angles_g(Sys s, BondList bl, AtomQ aq, Accum acc, const DParams<float>* __restrict__ P,
                           unsigned mask) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = gt / G;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  // no early exit: the group butterflies below span the whole warp
  const int nb = j < s.n ? bl.cnt[j] : 0;
  const bool act = nb >= 2;
  const int jj = act ? j : 0;
  const int tj = s.type[jj];
  const float* bo = (const float*)bl.bo;
  const float dang = aq.dang_f[jj], delta = aq.delta_f[jj];
  const float sbo2 = aq.sbo2_f[jj];
  const float wv = wbit<float>(mask, T_VAL), wp = wbit<float>(mask, T_PEN), wc = wbit<float>(mask, T_COA);
  const float pv5 = P->p_val5[tj];
  const float e6 = m_expc(P->p_val6 * dang);
  const float ex2 = m_exp(-P->p_val10 * (2.0f - sbo2));
  const float dth0_dsbo2 = ex2 * P->p_val10;
  float f9, df9;
  f9fun<float>(P->p_pen3, P->p_pen4, delta, f9, df9);
  float scoa, scoad;
  sig_pair<float>(P->p_coa2 * dang, scoa, scoad);
  float l_eval = 0, l_epen = 0, l_ecoa = 0, l_cdsbo = 0, l_cdd = 0;
  float l_fj[3] = {0, 0, 0}, l_w[6] = {0, 0, 0, 0, 0, 0};
  const int npair = act ? nb * (nb - 1) / 2 : 0;
  for (int p = sub; p < npair; p += G) {
    int a = 0, rem = p;
    while (rem >= nb - 1 - a) { rem -= nb - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const int ea = j * bl.cap + a, eb = j * bl.cap + b;
    const float BOa = bo[ea], BOb = bo[eb];
    if (!(BOa > P->thb_cut && BOb > P->thb_cut && BOa * BOb > P->thb_cutsq)) continue;
    const int i = bl.j[ea], k = bl.j[eb];
    const int ti = s.type[i], tk = s.type[k];
    const int t3 = (ti * MAXT + tj) * MAXT + tk;
    const Vec3<float> u = load_vec<float>(bl, ea), v = load_vec<float>(bl, eb);
    const float L1 = dot3(u, u), L2 = dot3(v, v);
    // theta = atan2(|u x v|, u.v): accurate at every angle; d theta/du = (u x n^)/|u|^2,
    // d theta/dv = (n^ x v)/|v|^2 with n^ = (u x v)/|u x v|
    const Vec3<float> nrm = cross_acc(u, v);
    const float nn = m_sqrt(dot3(nrm, nrm));
    const float th = m_atan2(nn, dot3(u, v));
    const bool cok = nn > float(0);
    // valence
    const float th00 = P->th00[t3];
    const float th0 = float(3.14159265358979323846) - th00 * (float(1) - ex2);
    const float pv3 = P->p_val3[tj], pv4 = P->p_val4[t3];
    const float pa = m_pow(BOa, pv4), pb = m_pow(BOb, pv4);
    const float ea7 = m_exp(-pv3 * pa), eb7 = m_exp(-pv3 * pb);
    const float f7a = -m_expm1(-pv3 * pa), f7b = -m_expm1(-pv3 * pb);
    const float df7a = ea7 * pv3 * pv4 * pa / BOa, df7b = eb7 * pv3 * pv4 * pb / BOb;
    // f8 = pv5 - (pv5 - 1)(2 + e6)/(1 + e6 + e7); with u = e6/den, v = e7/den:
    // d[(2 + e6)/den]/dDang = (2 p7 v - p6 u)/den + (p6 + p7) u v
    const float p7 = P->p_val7[t3];
    const float e7 = m_expc(-p7 * dang);
    const float den8 = float(1) + e6 + e7;
    const float u8 = e6 / den8, v8 = e7 / den8;
    const float f8 = pv5 - (pv5 - float(1)) * (float(2) / den8 + u8);
    const float df8 = -(pv5 - float(1)) * ((float(2) * p7 * v8 - P->p_val6 * u8) / den8 + (P->p_val6 + p7) * u8 * v8);
    const float pv1 = P->p_val1[t3], pv2 = P->p_val2[t3];
    const float D = th0 - th;
    const float exv = m_exp(-pv2 * D * D);
    const float gth = -m_expm1(-pv2 * D * D);
    const float Cv = f7a * f7b * f8 * pv1;
    const float ev = Cv * gth;
    const float dEdD = Cv * exv * float(2) * pv2 * D;          // d/dD of Cv (1 - e^{-pv2 D^2})
    const float dEv_dth = -dEdD;
    const float dEv_dsbo2 = dEdD * th00 * dth0_dsbo2;
    // penalty
    const float pp2 = P->p_pen2;
    const float ga = m_exp(-pp2 * (BOa - float(2)) * (BOa - float(2))), gb = m_exp(-pp2 * (BOb - float(2)) * (BOb - float(2)));
    const float ep = P->p_pen1[t3] * f9 * ga * gb;
    // coalition
    const float sbi = aq.sumbo_f[i] - BOa;
    const float sbk = aq.sumbo_f[k] - BOb;
    const float pc3 = P->p_coa3, pc4 = P->p_coa4;
    const float ec = P->p_coa1[t3] * scoa * m_exp(-pc3 * sbi * sbi) * m_exp(-pc3 * sbk * sbk) *
                 m_exp(-pc4 * (BOa - float(1.5)) * (BOa - float(1.5))) * m_exp(-pc4 * (BOb - float(1.5)) * (BOb - float(1.5)));
    l_eval += ev;
    l_epen += ep;
    l_ecoa += ec;
    // bond-order and Delta derivatives
    const float dBOa = wv * df7a * f7b * f8 * pv1 * gth + wp * ep * (float(-2) * pp2 * (BOa - float(2))) +
                   wc * ec * (float(2) * pc3 * sbi - float(2) * pc4 * (BOa - float(1.5)));
    const float dBOb = wv * f7a * df7b * f8 * pv1 * gth + wp * ep * (float(-2) * pp2 * (BOb - float(2))) +
                   wc * ec * (float(2) * pc3 * sbk - float(2) * pc4 * (BOb - float(1.5)));
    fix_add(bl.cdbo + ea, dBOa, s.err);
    fix_add(bl.cdbo + eb, dBOb, s.err);
    fix_add(aq.cddelta + i, wc * ec * (float(-2) * pc3 * sbi), s.err);
    fix_add(aq.cddelta + k, wc * ec * (float(-2) * pc3 * sbk), s.err);
    l_cdd += wv * f7a * f7b * df8 * pv1 * gth + wp * P->p_pen1[t3] * df9 * ga * gb +
             wc * (scoa > float(0) ? -ec * P->p_coa2 * scoad / scoa : float(0));
    l_cdsbo += wv * dEv_dsbo2;
    // geometry: E depends on cos(theta) only through the valence term
    if (cok) {
      const float gt = wv * dEv_dth / nn;
      const Vec3<float> cu = cross3(u, nrm), cv = cross3(nrm, v);
      const Vec3<float> gu = Vec3<float>{gt * cu.x / L1, gt * cu.y / L1, gt * cu.z / L1};
      const Vec3<float> gv = Vec3<float>{gt * cv.x / L2, gt * cv.y / L2, gt * cv.z / L2};
      force_add<float>(s, i, -gu.x, -gu.y, -gu.z);
      force_add<float>(s, k, -gv.x, -gv.y, -gv.z);
      l_fj[0] += gu.x + gv.x; l_fj[1] += gu.y + gv.y; l_fj[2] += gu.z + gv.z;
      vir_sub(l_w, gu, u);
      vir_sub(l_w, gv, v);
    }
  }
  constexpr int NVA = 14;   // 0-2 E_val, E_pen, E_coa; 3-5 F_j; 6-11 virial; 12 dE/dSBO2; 13 dE/dDelta
  float hi[NVA] = {l_eval, l_epen, l_ecoa, l_fj[0], l_fj[1], l_fj[2], l_w[0], l_w[1], l_w[2], l_w[3], l_w[4],
                   l_w[5], l_cdsbo, l_cdd};
  float lo[NVA];
#pragma unroll
  for (int q = 0; q < NVA; ++q) {
    lo[q] = 0.0f;
    GroupSum<float, G>::run(hi[q], lo[q]);
  }
  if (!act) return;
  // every total goes to a 2^-32 fixed-point accumulator through 32-bit conversions: no FP64
  // instruction (each would hold the SM's FP64 pipe for ~16 cycles)
  const float cdsbo = (hi[12] + lo[12]) * aq.dsbo2_f[j];   // dE/dSBO
  const float prod = aq.prodexp_f[j];
#pragma unroll
  for (int rnd = 0; rnd < (NVA + G - 1) / G; ++rnd) {
    const int q = sub + rnd * G;
    float h, l;
    lane_pick<NVA>(hi, lo, q, h, l);
    if (q < 3) {
      fix_add_ff(acc.efx + (size_t)(T_VAL + q) * s.n + j, h, l, s.err);
    } else if (q < 6) {
      fix_add_ff((q == 3 ? s.fx : q == 4 ? s.fy : s.fz) + j, h, l, s.err);
    } else if (q < 12) {
      fix_add_ff(acc.vfx + (size_t)(q - 6) * s.n + j, h, l, s.err);
    } else if (q == 13) {
      const float dsbo_dsum = -(1.0f - prod) * (1.0f + P->p_val8 * aq.dnlp_f[j]);
      fix_add_ff(aq.cddelta + j, h, l, s.err);
      fix_add(aq.cddelta + j, cdsbo * dsbo_dsum, s.err);
    }
  }
  // SBO depends on every bond of j: distribute dE/dSBO over j's row (FP32 terms)
  if (cdsbo != 0.0f) {
    const float cf = cdsbo, pf = prod, ff = aq.sbo_fac_f[j];
    for (int k = sub; k < nb; k += G) {
      const int e = j * bl.cap + k;
      const float b = bo[e];
      const float b2 = b * b, b4 = b2 * b2;
      fix_add(bl.cdbopi + e, cf, s.err);
      fix_add(bl.cdbopp + e, cf, s.err);
      fix_add(bl.cdbo + e, cf * pf * 8.0f * b4 * b2 * b * ff, s.err);
    }
  }
}

// One torsion + conjugation term (i-j-k-l over the central bond j-k, Sec. 3.3 "4-body"):
// energies and the derivatives with respect to BO_ij, BO_kl (fixed-point atomics on the bond
// entries), forces on i and l (atomics), and the contributions to the central bond's totals in
// v[18]: 0-2 F_j, 3 dE/dDelta_j, 4 E_tors, 5 E_conj, 6-11 virial, 12-14 F_k, 15 dE/dDelta_k,
// 16 dE/dBO_jk, 17 dE/dBOpi_jk. False (and nothing added) for a collinear i-j-k or j-k-l.
template <typename R>
struct TorsBond {              // quantities of the central bond j-k shared by its torsions
  R V1, V2, V3, pt1, pc1, pt2, pc2, BO2, xb, ex, g2, dg2, h2, df11, L2, l2;
  Vec3<R> u2;
  int j, k, ejk, code;
};

template <typename R>
__device__ __forceinline__ void tors_bond(const Sys& s, const BondList& bl, const AtomQ& aq, const DParams<R>* P, int j,
                                          int k, int ejk, TorsBond<R>& b) {
  const R* bo = (const R*)bl.bo;
  const R* bo_pi = (const R*)bl.bo_pi;
  const int pt = s.type[j] * MAXT + s.type[k];
  b.V1 = P->V1[pt]; b.V2 = P->V2[pt]; b.V3 = P->V3[pt]; b.pt1 = P->p_tor1[pt]; b.pc1 = P->p_cot1[pt];
  b.pt2 = P->p_tor2; b.pc2 = P->p_cot2;
  b.BO2 = bo[ejk];
  const R BOpi2 = bo_pi[ejk];
  R Dsum;
  if constexpr (sizeof(R) == 4) Dsum = aq.dang_f[j] + aq.dang_f[k];
  else Dsum = (R)(aq.dang[j] + aq.dang[k]);
  R f11, df11;
  f9fun<R>(P->p_tor3, P->p_tor4, Dsum, f11, df11);
  b.df11 = df11;
  b.xb = R(2) - BOpi2 - f11;
  b.ex = m_exp(b.pt1 * b.xb * b.xb);
  b.g2 = -m_expm1(-b.pt2 * b.BO2);
  b.dg2 = b.pt2 * m_exp(-b.pt2 * b.BO2);
  b.h2 = m_exp(-b.pc2 * (b.BO2 - R(1.5)) * (b.BO2 - R(1.5)));
  b.u2 = load_vec<R>(bl, ejk);
  b.L2 = dot3(b.u2, b.u2);
  b.l2 = m_sqrt(b.L2);
  b.j = j; b.k = k; b.ejk = ejk; b.code = bl.s[ejk];
}

template <typename R>
__device__ __forceinline__ bool torsion_term(const Sys& s, const BondList& bl, const TorsBond<R>& b, R wt, R wcj,
                                            int ea, int ec, int i, int l, R BO1, R BO3, R* v) {
  const R V1 = b.V1, V2 = b.V2, V3 = b.V3, pt1 = b.pt1, pc1 = b.pc1, pt2 = b.pt2, pc2 = b.pc2;
  const R BO2 = b.BO2, xb = b.xb, ex = b.ex, g2 = b.g2, dg2 = b.dg2, h2 = b.h2, df11 = b.df11;
  const R L2 = b.L2, l2 = b.l2;
  const Vec3<R> u2 = b.u2;
  const Vec3<R> u1 = load_vec<R>(bl, ea), u3 = load_vec<R>(bl, ec);
  // Well-conditioned torsion geometry: n1 = u1 x u2, n2 = u3 x u2, A = |n1|, B = |n2|,
  // P = n1.n2, V = u3.n1 (L2 V^2 = A^2 B^2 - P^2), D0 = l1 l2^2 l3. Then
  //   s1 s2 = A B / D0 = S,  s1 s2 cos w = P / D0 = C,  s1 s2 cos^3 w = P^3/(A^2 B^2 D0) = M,
  //   s1 s2 (1 - cos^2 w) = V^2 / (A B l1 l3) = Y,
  //   E_tors = f10 [V1 (S + C)/2 + V2 e Y + V3 (S + 4M - 3C)/2],  E_conj = K (1 - Y).
  const Vec3<R> n1 = cross_acc(u1, u2), n2 = cross_acc(u3, u2);
  const R A2 = dot3(n1, n1), B2 = dot3(n2, n2);
  const R L1 = dot3(u1, u1), L3 = dot3(u3, u3);
  const R l1 = m_sqrt(L1), l3 = m_sqrt(L3);
  const R Am = m_sqrt(A2), Bm = m_sqrt(B2);
  if (!(Am > R(1e-10) * l1 * l2 && Bm > R(1e-10) * l2 * l3)) return false;   // collinear: sin th ~ 0
  const R Pn = dot3(n1, n2);
  const R Vt = dot3(u3, n1);
  const R D0 = l1 * L2 * l3;
  const R cw = rclamp(Pn / (Am * Bm), R(-1), R(1));
  const R S = Am * Bm / D0, Cc = Pn / D0, M = cw * cw * Cc, Y = Vt * Vt / (Am * Bm * l1 * l3);
  // energy
  const R g1 = -m_expm1(-pt2 * BO1), g3 = -m_expm1(-pt2 * BO3);
  const R dg1 = pt2 * m_exp(-pt2 * BO1), dg3 = pt2 * m_exp(-pt2 * BO3);
  const R f10 = g1 * g2 * g3;
  const R Tsum = R(0.5) * V1 * (S + Cc) + V2 * ex * Y + R(0.5) * V3 * (S + R(4) * M - R(3) * Cc);
  const R h1 = m_exp(-pc2 * (BO1 - R(1.5)) * (BO1 - R(1.5)));
  const R h3 = m_exp(-pc2 * (BO3 - R(1.5)) * (BO3 - R(1.5)));
  const R K = pc1 * h1 * h2 * h3;
  const R et = f10 * Tsum;
  const R ecj = K * (R(1) - Y);
  v[4] += et;
  v[5] += ecj;
  // non-geometric derivatives
  const R dBO1 = wt * dg1 * g2 * g3 * Tsum + wcj * ecj * (R(-2) * pc2 * (BO1 - R(1.5)));
  const R dBO3 = wt * g1 * g2 * dg3 * Tsum + wcj * ecj * (R(-2) * pc2 * (BO3 - R(1.5)));
  const R dBO2 = wt * g1 * dg2 * g3 * Tsum + wcj * ecj * (R(-2) * pc2 * (BO2 - R(1.5)));
  const R dTdx = V2 * Y * ex * pt1 * R(2) * xb;   // d Tsum / d xb
  const R dpi = wt * f10 * dTdx * R(-1);
  const R dD = wt * f10 * dTdx * (-df11);
  fix_add(bl.cdbo + ea, dBO1, s.err);
  fix_add(bl.cdbo + ec, dBO3, s.err);
  v[16] += dBO2;
  v[17] += dpi;
  v[3] += dD;
  v[15] += dD;
  // geometric derivatives through (A, B, P, V, l1, l2, l3)
  const R dES = wt * f10 * R(0.5) * (V1 + V3);
  const R dEC = wt * f10 * (R(0.5) * V1 - R(1.5) * V3);
  const R dEM = wt * f10 * R(2) * V3;
  const R dEY = wt * f10 * V2 * ex - wcj * K;
  const R gA = (dES * S - R(2) * dEM * M - dEY * Y) / Am;
  const R gB = (dES * S - R(2) * dEM * M - dEY * Y) / Bm;
  const R gP = (dEC + dEM * R(3) * cw * cw) / D0;
  const R gV = dEY * R(2) * Vt / (Am * Bm * l1 * l3);
  const R T0 = dES * S + dEC * Cc + dEM * M;
  const R gl1 = -(T0 + dEY * Y) / L1;             // per unit of u1 (d l1 / d u1 = u1 / l1)
  const R gl2 = R(-2) * T0 / L2;
  const R gl3 = -(T0 + dEY * Y) / L3;
  const R iA = gA / Am, iB = gB / Bm;
  // dA/du1 = (u2 x n1)/A, dA/du2 = (n1 x u1)/A, dB/du3 = (u2 x n2)/B, dB/du2 = (n2 x u3)/B
  // dP/du1 = u2 x n2, dP/du2 = n2 x u1 + n1 x u3, dP/du3 = u2 x n1
  // dV/du1 = u2 x u3, dV/du2 = u3 x u1, dV/du3 = n1
  const Vec3<R> u2n1 = cross3(u2, n1), u2n2 = cross3(u2, n2), u2u3 = cross3(u2, u3);
  const Vec3<R> n1u1 = cross3(n1, u1), n2u3 = cross3(n2, u3), n2u1 = cross3(n2, u1), n1u3 = cross3(n1, u3);
  const Vec3<R> u3u1 = cross3(u3, u1);
  Vec3<R> gg1, gg2, gg3;
  gg1.x = iA * u2n1.x + gP * u2n2.x + gV * u2u3.x + gl1 * u1.x;
  gg1.y = iA * u2n1.y + gP * u2n2.y + gV * u2u3.y + gl1 * u1.y;
  gg1.z = iA * u2n1.z + gP * u2n2.z + gV * u2u3.z + gl1 * u1.z;
  gg2.x = iA * n1u1.x + iB * n2u3.x + gP * (n2u1.x + n1u3.x) + gV * u3u1.x + gl2 * u2.x;
  gg2.y = iA * n1u1.y + iB * n2u3.y + gP * (n2u1.y + n1u3.y) + gV * u3u1.y + gl2 * u2.y;
  gg2.z = iA * n1u1.z + iB * n2u3.z + gP * (n2u1.z + n1u3.z) + gV * u3u1.z + gl2 * u2.z;
  gg3.x = iB * u2n2.x + gP * u2n1.x + gV * n1.x + gl3 * u3.x;
  gg3.y = iB * u2n2.y + gP * u2n1.y + gV * n1.y + gl3 * u3.y;
  gg3.z = iB * u2n2.z + gP * u2n1.z + gV * n1.z + gl3 * u3.z;
  force_add<R>(s, i, -gg1.x, -gg1.y, -gg1.z);
  force_add<R>(s, l, -gg3.x, -gg3.y, -gg3.z);
  v[0] += gg1.x + gg2.x; v[1] += gg1.y + gg2.y; v[2] += gg1.z + gg2.z;
  v[12] += gg3.x - gg2.x; v[13] += gg3.y - gg2.y; v[14] += gg3.z - gg2.z;
  vir_sub(v + 6, gg1, u1);
  vir_sub(v + 6, gg2, u2);
  vir_sub(v + 6, gg3, u3);
  return true;
}

template <typename R, int TG>
__global__ void __launch_bounds__(128) k_torsions(Sys s, BondList bl, AtomQ aq, Accum acc,
                                                   const DParams<R>* __restrict__ P, unsigned mask) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (TG - 1);
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int ncanon = *bl.ncanon;
  const R* bo = (const R*)bl.bo;
  const R* bo_pi = (const R*)bl.bo_pi;
  const R wt = wbit<R>(mask, T_TORS), wcj = wbit<R>(mask, T_CONJ);
  // warp-uniform loop: 32/TG central bonds per warp and pass
  for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / TG); base < ncanon;
       base += nwarps * (32 / TG)) {
    const int t = base + lane / TG;
    int j = 0, k = 0, ejk = 0, ekj = 0, nbj = 0, nbk = 0, ntot = 0, codejk = 13;
    if (t < ncanon) {
      ejk = bl.canon[t];
      j = ejk / bl.cap;
      k = bl.j[ejk];
      codejk = bl.s[ejk];
      nbj = bl.cnt[j];
      nbk = bl.cnt[k];
      ekj = bl.mirror[ejk];
      if (nbj >= 2 && nbk >= 2 && ekj / bl.cap == k && bo[ejk] > P->thb_cut) ntot = (nbj - 1) * (nbk - 1);
    }
    // per-lane partials: 0-2 F_j, 3 dE/dDelta_j, 4 E_tors, 5 E_conj, 6-11 virial (at j),
    // 12-14 F_k, 15 dE/dDelta_k, 16 dE/dBO_jk, 17 dE/dBOpi_jk
    constexpr int NV = 18;
    R v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = R(0);
    if (ntot > 0) {
      TorsBond<R> tb;
      tors_bond<R>(s, bl, aq, P, j, k, ejk, tb);
      const R BO2 = tb.BO2;
      int sjk[3];
      shift_decode(codejk, sjk[0], sjk[1], sjk[2]);
      for (int p = sub; p < ntot; p += TG) {
        const int ia = p / (nbk - 1), ic = p % (nbk - 1);
        const int ea = j * bl.cap + ia + (j * bl.cap + ia >= ejk ? 1 : 0);
        int ec = k * bl.cap + ic;
        if (ec >= ekj) ++ec;
        const int i = bl.j[ea], l = bl.j[ec];
        if (i == l) {
          int si[3], sl[3];
          shift_decode(bl.s[ea], si[0], si[1], si[2]);
          shift_decode(bl.s[ec], sl[0], sl[1], sl[2]);
          if (si[0] == sjk[0] + sl[0] && si[1] == sjk[1] + sl[1] && si[2] == sjk[2] + sl[2]) continue;
        }
        const R BO1 = bo[ea], BO3 = bo[ec];
        if (!(BO1 * BO2 * BO3 > P->thb_cut)) continue;
        if (!torsion_term<R>(s, bl, tb, wt, wcj, ea, ec, i, l, BO1, BO3, v)) continue;
      }
    }
    // group totals (all lanes take part: the shuffles span the whole warp), then lane q of
    // the group adds values q, q + TG, q + 2 TG
    R hi[NV], lo[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      hi[q] = v[q];
      lo[q] = R(0);
      GroupSum<R, TG>::run(hi[q], lo[q]);
    }
    if (ntot > 0) {
#pragma unroll
      for (int rnd = 0; rnd < (NV + TG - 1) / TG; ++rnd) {
        const int q = sub + rnd * TG;
        R h = R(0), l = R(0);
#pragma unroll
        for (int c = 0; c < NV; ++c)
          if (c == q) {
            h = hi[c];
            l = lo[c];
          }
        unsigned long long* dst = nullptr;
        if (q < 3) dst = (q == 0 ? s.fx : q == 1 ? s.fy : s.fz) + j;
        else if (q == 3) dst = aq.cddelta + j;
        else if (q < 6) dst = acc.efx + (size_t)(T_TORS + q - 4) * s.n + j;
        else if (q < 12) dst = acc.vfx + (size_t)(q - 6) * s.n + j;
        else if (q < 15) dst = (q == 12 ? s.fx : q == 13 ? s.fy : s.fz) + k;
        else if (q == 15) dst = aq.cddelta + k;
        else if (q == 16) dst = bl.cdbo + ejk;
        else if (q == 17) dst = bl.cdbopi + ejk;
        if (dst) GroupSum<R, TG>::add(dst, h, l, s.err);
      }
    }
  }
}

// Mixed path, candidate compaction: a warp takes NB = 32 / TG central bonds per pass; the TG
// lanes of each group test their bond's (i, l) candidates with the cheap threshold and the
// passing ones are appended (ballot order) to a per-warp queue in shared memory; whenever 32
// are queued all lanes evaluate one each (torsion_term), so the heavy arithmetic runs on full
// warps instead of on the ~40 % of lanes whose candidate passed. A lane adds its term's
// contributions to the central bond's atoms and entries directly to the global 2^-32 fixed-
// point accumulators (integer atomics without a return value: exact, so their order does not
// matter and the sums are deterministic; no per-bond pre-sum is needed). Launch bounds of
// 7 blocks of 128 per SM cap it at 72 registers (94 uncapped; 12 bytes of spills): 28 warps
// per SM instead of 20 (1,039,360 atoms: 1.22 -> 1.08 ms). Forces, energies, virial and a
// 20-step trajectory of the capped build were bitwise equal over three runs: every queued
// term is evaluated by the one call site of the torsion arithmetic.
template <int TG>
__global__ void __launch_bounds__(128, 7) k_torsions_q(Sys s, BondList bl, AtomQ aq, Accum acc,
                                                     const DParams<float>* __restrict__ P, unsigned mask) {
  constexpr int NB = 32 / TG, NV = 18, QCAP = 64, WPB = 4;
  __shared__ TorsBond<float> sb[WPB][NB];
  __shared__ int4 sq[WPB][QCAP];
  __shared__ int sslot[WPB][QCAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sub = lane & (TG - 1), g = lane / TG;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int ncanon = *bl.ncanon;
  const float* bo = (const float*)bl.bo;
  const float wt = wbit<float>(mask, T_TORS), wcj = wbit<float>(mask, T_CONJ);
  const float thb = P->thb_cut;
  const unsigned below = (1u << lane) - 1u;

  auto batch = [&](int nact) {
    if (lane < nact) {
      const int4 e = sq[w][lane];
      const int gg = sslot[w][lane];
      float v[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] = 0.f;
      if (torsion_term<float>(s, bl, sb[w][gg], wt, wcj, e.x, e.y, e.z, e.w, bo[e.x], bo[e.y], v)) {
        const int bj = sb[w][gg].j, bk = sb[w][gg].k, be = sb[w][gg].ejk;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          unsigned long long* dst;
          if (c < 3) dst = (c == 0 ? s.fx : c == 1 ? s.fy : s.fz) + bj;
          else if (c == 3) dst = aq.cddelta + bj;
          else if (c < 6) dst = acc.efx + (size_t)(T_TORS + c - 4) * s.n + bj;
          else if (c < 12) dst = acc.vfx + (size_t)(c - 6) * s.n + bj;
          else if (c < 15) dst = (c == 12 ? s.fx : c == 13 ? s.fy : s.fz) + bk;
          else if (c == 15) dst = aq.cddelta + bk;
          else if (c == 16) dst = bl.cdbo + be;
          else dst = bl.cdbopi + be;
          fix_add(dst, v[c], s.err);
        }
      }
    }
    __syncwarp();
  };

  for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * NB; base < ncanon; base += nwarps * NB) {
    const int t = base + g;
    int j = 0, k = 0, ejk = 0, ekj = 0, nbk = 0, ntot = 0;
    if (t < ncanon) {
      ejk = bl.canon[t];
      j = ejk / bl.cap;
      k = bl.j[ejk];
      const int nbj = bl.cnt[j];
      nbk = bl.cnt[k];
      ekj = bl.mirror[ejk];
      if (nbj >= 2 && nbk >= 2 && ekj / bl.cap == k && bo[ejk] > thb) ntot = (nbj - 1) * (nbk - 1);
    }
    if (ntot > 0 && sub == 0) tors_bond<float>(s, bl, aq, P, j, k, ejk, sb[w][g]);
    __syncwarp();
    const float BO2 = ntot > 0 ? bo[ejk] : 0.f;
    int sjk[3] = {0, 0, 0};
    if (ntot > 0) shift_decode(bl.s[ejk], sjk[0], sjk[1], sjk[2]);
    const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)((ntot + TG - 1) / TG));
    int qn = 0;
    // rounds of candidate tests, then one more pass that only flushes the queue: every
    // queued candidate is evaluated by the one batch() call below, whichever pass or queue
    // position it lands in (the canonical-bond order, and so the queues, vary from run to
    // run: canon is filled by an atomic append)
    for (int rd = 0; rd <= rounds; ++rd) {
      const int p = rd * TG + sub;
      bool pass = false;
      int ea = 0, ec = 0, i = 0, l = 0;
      if (rd < rounds && p < ntot) {
        const int ia = p / (nbk - 1), ic = p % (nbk - 1);
        ea = j * bl.cap + ia + (j * bl.cap + ia >= ejk ? 1 : 0);
        ec = k * bl.cap + ic;
        if (ec >= ekj) ++ec;
        i = bl.j[ea];
        l = bl.j[ec];
        pass = true;
        if (i == l) {
          int si[3], sl[3];
          shift_decode(bl.s[ea], si[0], si[1], si[2]);
          shift_decode(bl.s[ec], sl[0], sl[1], sl[2]);
          if (si[0] == sjk[0] + sl[0] && si[1] == sjk[1] + sl[1] && si[2] == sjk[2] + sl[2]) pass = false;
        }
        if (pass) pass = bo[ea] * BO2 * bo[ec] > thb;
      }
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        const int pos = qn + __popc(m & below);
        sq[w][pos] = make_int4(ea, ec, i, l);
        sslot[w][pos] = g;
      }
      qn += __popc(m);
      __syncwarp();
      // a full batch of 32 while testing, whatever is left on the flushing pass (qn < 32
      // then); qn, rd and rounds are warp-uniform
      const int nact = rd < rounds ? (qn >= 32 ? 32 : 0) : qn;
      if (nact > 0) {
        batch(nact);
        const int left = qn - nact;
        int4 e = make_int4(0, 0, 0, 0);
        int gs = 0;
        if (lane < left) { e = sq[w][32 + lane]; gs = sslot[w][32 + lane]; }
        __syncwarp();
        if (lane < left) { sq[w][lane] = e; sslot[w][lane] = gs; }
        __syncwarp();
        qn = left;
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ hydrogen bonds
template <typename R>
__global__ void k_hbonds(Sys s, BondList bl, HbList hl, Accum acc, const DParams<R>* __restrict__ P,
                         unsigned mask) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= s.n) return;
  const int tj = s.type[j];
  if (P->hb[tj] != 1) return;
  const int nb = bl.cnt[j], nz = hl.cnt[j];
  const R* bo = (const R*)bl.bo;
  const R wh = wbit<R>(mask, T_HB);
  const int r = s.rep[j];
  R l_ehb = 0, l_fj[3] = {0, 0, 0}, l_w[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < nb; ++a) {
    const int ea = j * bl.cap + a;
    const int x = bl.j[ea];
    const int tx = s.type[x];
    const R BO = bo[ea];
    if (P->hb[tx] != 2 || !(BO >= P->hb_bo_min)) continue;
    const int codea = bl.s[ea];
    const Vec3<R> u = load_vec<R>(bl, ea);
    const R Lu = dot3(u, u), lu = m_sqrt(Lu);
    R l_cdb = 0, l_fx[3] = {0, 0, 0};
    for (int zz = lane; zz < nz; zz += 32) {
      const int ez = j * hl.cap + zz;
      const int z = hl.j[ez];
      const int codez = hl.s[ez];
      if (z == x && codez == codea) continue;
      const int tz = s.type[z];
      const int pt = tx * MAXT + tz;
      Vec3<R> v;
      PairVec<R>::get(s, j, z, codez, r, v.x, v.y, v.z);
      const R Lv = dot3(v, v), lv = m_sqrt(Lv), A = dot3(u, v);
      const R cr = A / (lu * lv);
      const bool cok = cr > R(-1) && cr < R(1);
      const R c = rclamp(cr, R(-1), R(1));
      const R r0 = P->r0hb[pt];
      const R eb = m_exp(-P->p_hb2[pt] * BO);
      const R er = m_exp(-P->p_hb3[pt] * (r0 / lv + lv / r0 - R(2)));
      const R hs = R(0.5) * (R(1) - c);
      const R s4 = hs * hs;
      const R ph1 = P->p_hb1[pt];
      const R omeb = -m_expm1(-P->p_hb2[pt] * BO);
      const R e = ph1 * omeb * er * s4;
      l_ehb += e;
      l_cdb += wh * ph1 * P->p_hb2[pt] * eb * er * s4;
      const R dEdr = wh * e * (-P->p_hb3[pt]) * (-r0 / Lv + R(1) / r0);
      const R dEdc = cok ? wh * ph1 * omeb * er * (-hs) : R(0);
      const R dEdA = dEdc / (lu * lv);
      const R dEdLu = dEdc * (-c / (R(2) * Lu));
      const R dEdLv = dEdc * (-c / (R(2) * Lv)) + dEdr / (R(2) * lv);
      const Vec3<R> gu = lin2(dEdA, v, R(2) * dEdLu, u);
      const Vec3<R> gv = lin2(dEdA, u, R(2) * dEdLv, v);
      force_add<R>(s, z, -gv.x, -gv.y, -gv.z);
      l_fx[0] -= gu.x; l_fx[1] -= gu.y; l_fx[2] -= gu.z;
      l_fj[0] += gu.x + gv.x; l_fj[1] += gu.y + gv.y; l_fj[2] += gu.z + gv.z;
      vir_sub(l_w, gu, u);
      vir_sub(l_w, gv, v);
    }
    if constexpr (sizeof(R) == 4) {
      constexpr int NVX = 4;   // 0 dE/dBO_jx, 1-3 F_x
      float hi[NVX] = {l_cdb, l_fx[0], l_fx[1], l_fx[2]};
      float lo[NVX];
#pragma unroll
      for (int q = 0; q < NVX; ++q) {
        lo[q] = 0.0f;
        warp_sum_ff2(hi[q], lo[q]);
      }
      float h, l;
      lane_pick<NVX>(hi, lo, lane, h, l);
      if (lane < NVX)
        fix_add_ff(lane == 0 ? bl.cdbo + ea : lane == 1 ? s.fx + x : lane == 2 ? s.fy + x : s.fz + x, h, l, s.err);
    } else {
      const double cdb = warp_sum_d(l_cdb);
      double fx[3];
      for (int q = 0; q < 3; ++q) fx[q] = warp_sum_d(l_fx[q]);
      if (lane == 0) {
        fix_add(bl.cdbo + ea, cdb, s.err);
        force_add<double>(s, x, fx[0], fx[1], fx[2]);
      }
    }
  }
  if constexpr (sizeof(R) == 4) {
    constexpr int NVJ = 10;   // 0 E_hb; 1-3 F_j; 4-9 virial
    float hi[NVJ] = {l_ehb, l_fj[0], l_fj[1], l_fj[2], l_w[0], l_w[1], l_w[2], l_w[3], l_w[4], l_w[5]};
    float lo[NVJ];
#pragma unroll
    for (int q = 0; q < NVJ; ++q) {
      lo[q] = 0.0f;
      warp_sum_ff2(hi[q], lo[q]);
    }
    float h, l;
    lane_pick<NVJ>(hi, lo, lane, h, l);
    if (lane == 0) {
      fix_add_ff(acc.efx + (size_t)T_HB * s.n + j, h, l, s.err);
    } else if (lane < 4) {
      fix_add_ff(lane == 1 ? s.fx + j : lane == 2 ? s.fy + j : s.fz + j, h, l, s.err);
    } else if (lane < NVJ) {
      fix_add_ff(acc.vfx + (size_t)(lane - 4) * s.n + j, h, l, s.err);
    }
  } else {
    const double ehb = warp_sum_d(l_ehb);
    double fj[3], w[6];
    for (int q = 0; q < 3; ++q) fj[q] = warp_sum_d(l_fj[q]);
    for (int q = 0; q < 6; ++q) w[q] = warp_sum_d(l_w[q]);
    if (lane == 0) {
      acc.e[T_HB * s.n + j] = ehb;
      force_add<double>(s, j, fj[0], fj[1], fj[2]);
      for (int q = 0; q < 6; ++q) acc.vir[q * s.n + j] += w[q];
    }
  }
}

}  // namespace

namespace rx {

template <typename R> void bo_correct(const Launch& L, Sys s, BondList b, AtomQ a, const DParams<R>* P) {
  // two threads per atom: about one pass over the canonical bonds of molecular systems (the
  // loop strides over any more)
  k_bo_correct<R><<<grid_for(2LL * s.n, 128), 128, 0, L.st>>>(s, b, a, P);
  *L.count += 1;
}
template <typename R>
void atom_terms(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P, unsigned mask) {
  k_atom_terms<R><<<grid_for(s.n, 128), 128, 0, L.st>>>(s, b, a, acc, P, mask);
  *L.count += 1;
}
template <typename R>
void over_under_bond(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P, unsigned mask) {
  k_over_under_bond<R><<<grid_for(s.n, 128), 128, 0, L.st>>>(s, b, a, acc, P, mask);
  *L.count += 1;
}
template <typename R> void s_gather(const Launch& L, Sys s, BondList b, AtomQ a) {
  k_s_gather<R><<<grid_for(s.n, 128), 128, 0, L.st>>>(s, b, a);
  *L.count += 1;
}
template <typename R>
void angles(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P, unsigned mask) {
  const int bs = L.t().ang_block;
  const int g = L.t().ang_lanes;
  if constexpr (sizeof(R) == 4) {
    const unsigned grid = grid_for((long long)s.n * g, bs);
    if (g == 4) k_angles_g<4><<<grid, bs, 0, L.st>>>(s, b, a, acc, P, mask);
    else if (g == 8) k_angles_g<8><<<grid, bs, 0, L.st>>>(s, b, a, acc, P, mask);
    else if (g == 16) k_angles_g<16><<<grid, bs, 0, L.st>>>(s, b, a, acc, P, mask);
    else k_angles_g<32><<<grid, bs, 0, L.st>>>(s, b, a, acc, P, mask);
  } else {
    k_angles<R><<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, b, a, acc, P, mask);
  }
  *L.count += 1;
}
template <typename R>
void torsions(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P, unsigned mask) {
  // one group of lanes per central bond; about one central bond per atom in molecular
  // systems: the grid covers n central bonds in one pass and loops beyond that
  const int tg = L.t().tors_lanes;
  const unsigned grid = grid_for((long long)s.n * tg, 128);
  if constexpr (sizeof(R) == 4) {
    if (tg == 1) k_torsions_q<1><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
    else if (tg == 2) k_torsions_q<2><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
    else if (tg == 8) k_torsions_q<8><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
    else k_torsions_q<4><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
  } else {
    if (tg == 2) k_torsions<R, 2><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
    else if (tg == 8) k_torsions<R, 8><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
    else k_torsions<R, 4><<<grid, 128, 0, L.st>>>(s, b, a, acc, P, mask);
  }
  *L.count += 1;
}
template <typename R>
void hbonds(const Launch& L, Sys s, BondList b, HbList h, Accum acc, const DParams<R>* P, unsigned mask) {
  const int bs = L.t().hb_block;
  k_hbonds<R><<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, b, h, acc, P, mask);
  *L.count += 1;
}

#define INST(R)                                                                                           \
  template void bo_correct<R>(const Launch&, Sys, BondList, AtomQ, const DParams<R>*);                    \
  template void atom_terms<R>(const Launch&, Sys, BondList, AtomQ, Accum, const DParams<R>*, unsigned);   \
  template void over_under_bond<R>(const Launch&, Sys, BondList, AtomQ, Accum, const DParams<R>*, unsigned); \
  template void s_gather<R>(const Launch&, Sys, BondList, AtomQ);                                         \
  template void angles<R>(const Launch&, Sys, BondList, AtomQ, Accum, const DParams<R>*, unsigned);       \
  template void torsions<R>(const Launch&, Sys, BondList, AtomQ, Accum, const DParams<R>*, unsigned);     \
  template void hbonds<R>(const Launch&, Sys, BondList, HbList, Accum, const DParams<R>*, unsigned);
INST(double)
INST(float)
}  // namespace rx

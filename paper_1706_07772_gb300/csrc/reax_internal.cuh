// Internal declarations of the ReaxFF GB300 library: device data layout, device
// helpers (fixed-point accumulation, warp reductions, bounded grid barrier) and the
// kernel launch entry points shared between translation units.
//
// Layout in HBM (all per-atom data structure-of-arrays, atoms in input order):
//   positions/velocities   double x[n], y[n], z[n], vx.., with float copies xf.. for
//                          list filtering
//   far list (ELL)         row i at [i*cap_far, i*cap_far + far_cnt[i]): int32 j,
//                          uint8 image-shift code, H value (QEq matrix entry, type R)
//   bond list (ELL)        row i at [i*cap_bond, ...): j, shift, mirror entry index,
//                          geometry, BO' parts and their r-derivatives, corrected BO
//                          parts and the correction derivatives (type R), dE/dBO
//                          accumulators (int64 fixed point)
//   H-bond list (ELL)      row i (H atoms only) at [i*cap_hb, ...): j, shift
// Forces, dE/dBO and dE/dDelta are accumulated as int64 fixed point (2^-32 quanta):
// integer addition is associative, so every result is bitwise reproducible.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "reaxff.h"

#define MAXT REAXFF_MAXT
#define NTERMS REAXFF_NTERMS

enum { T_BOND = 0, T_LP, T_OVER, T_UNDER, T_VAL, T_PEN, T_COA, T_TORS, T_CONJ, T_HB, T_VDW,
       T_COUL, T_POL };

// error flag bits (device-side, read by the host after a stage)
enum { ERR_CAP_FAR = 1, ERR_CAP_BOND = 2, ERR_CAP_HB = 4, ERR_TIMEOUT = 8, ERR_NAN = 16,
       ERR_CG = 32, ERR_CAP_NEAR = 64, ERR_CAP_CAND = 128, ERR_CAP_DESC = 256 };

constexpr double FIX_SCALE = 4294967296.0;         // 2^32
constexpr double FIX_INV = 1.0 / 4294967296.0;
constexpr double FIX_LIMIT = 1.0e9;                // |value| beyond this -> ERR_NAN

// ------------------------------------------------------------------ parameters
template <typename R>
struct DParams {
  int nt;
  int hb[MAXT];
  R mass[MAXT], val[MAXT], vale[MAXT], valboc[MAXT], valang[MAXT], p_lp2[MAXT], p_ovun2[MAXT],
      p_ovun5[MAXT], p_val3[MAXT], p_val5[MAXT], chi[MAXT], eta[MAXT];
  R r0s[MAXT * MAXT], r0p[MAXT * MAXT], r0pp[MAXT * MAXT], p_bo1[MAXT * MAXT], p_bo2[MAXT * MAXT],
      p_bo3[MAXT * MAXT], p_bo4[MAXT * MAXT], p_bo5[MAXT * MAXT], p_bo6[MAXT * MAXT],
      p_boc3[MAXT * MAXT], p_boc4[MAXT * MAXT], p_boc5[MAXT * MAXT], ovc[MAXT * MAXT],
      v13[MAXT * MAXT], De_s[MAXT * MAXT], De_p[MAXT * MAXT], De_pp[MAXT * MAXT],
      p_be1[MAXT * MAXT], p_be2[MAXT * MAXT], p_ovun1[MAXT * MAXT], vdw_D[MAXT * MAXT],
      vdw_rv[MAXT * MAXT], vdw_alpha[MAXT * MAXT], vdw_gw_pow[MAXT * MAXT],  // gw^-p_vdW1
      gamma_m3[MAXT * MAXT];                                                 // gamma^-3
  R th00[MAXT * MAXT * MAXT], p_val1[MAXT * MAXT * MAXT], p_val2[MAXT * MAXT * MAXT],
      p_val4[MAXT * MAXT * MAXT], p_val7[MAXT * MAXT * MAXT], p_pen1[MAXT * MAXT * MAXT],
      p_coa1[MAXT * MAXT * MAXT];
  R r0s_lo[MAXT * MAXT], r0p_lo[MAXT * MAXT], r0pp_lo[MAXT * MAXT];   // r0 - R(r0) (float-float)
  R lr0s[MAXT * MAXT], lr0p[MAXT * MAXT], lr0pp[MAXT * MAXT];         // log r0 (0 where r0 <= 0)
  // bond membership as a distance: BO'(r) >= bo_cut exactly when r <= bcut (each BO' term
  // decreases with r); bcut as double and float-float; bcut_ok = 0 where that does not hold
  // for the parameters (then membership is decided in FP64 every time)
  double bcut[MAXT * MAXT];
  float bcut_h[MAXT * MAXT], bcut_l[MAXT * MAXT];
  int bcut_ok[MAXT * MAXT];
  R V1[MAXT * MAXT], V2[MAXT * MAXT], V3[MAXT * MAXT], p_tor1[MAXT * MAXT], p_cot1[MAXT * MAXT];
  R r0hb[MAXT * MAXT], p_hb1[MAXT * MAXT], p_hb2[MAXT * MAXT], p_hb3[MAXT * MAXT];
  // far-pair constants per type pair, rounded once from FP64 (mixed-path nonbonded):
  // [gw^-p_vdW1, alpha log2(e), 1/r_vdW, D, gamma^-3, -D alpha / r_vdW, 0, 0]
  alignas(16) R nbf[MAXT * MAXT * 8];
  R p_boc1, p_boc2, p_lp1, p_ovun3, p_ovun4, p_ovun6, p_ovun7, p_ovun8, p_val6, p_val8, p_val9,
      p_val10, p_pen2, p_pen3, p_pen4, p_coa2, p_coa3, p_coa4, p_tor2, p_tor3, p_tor4, p_cot2,
      p_vdW1, k_e;
  // options needed inside kernels
  R r_nb, r_bond, r_hb, bo_cut, thb_cut, thb_cutsq, hb_bo_min;
};

// ------------------------------------------------------------------ device views
struct Sys {                   // per-atom and per-replica state
  int n, nrep;
  const int* type;
  const int* rep;              // replica of each atom
  const double* box;           // [nrep*3]
  const int64_t* rep_off;      // [nrep+1]
  const float* boxh;           // [nrep*3] float(L)
  const float* boxl;           // [nrep*3] float(L - float(L))
  double *x, *y, *z;
  float *xh, *yh, *zh;         // float(x)
  float *xl, *yl, *zl;         // float(x - float(x))
  double *vx, *vy, *vz;
  unsigned long long *fx, *fy, *fz;   // fixed-point force accumulators
  double* q;
  float* qf;                   // FP32 copy of q (mixed-path nonbonded)
  float4* ph;                  // packed FP32 pair records (mixed path; may be null):
  float4* pl;                  //   ph = (x_hi, y_hi, z_hi, q), pl = (x_lo, y_lo, z_lo, type bits)
  int* err;
  int* img;                    // [3n] box crossings since the last candidate-list build
  double* xb;                  // [3n] wrapped positions at the last candidate-list build
  int* rebuild;                // device flag: rebuild the candidate list this step
};

// Verlet-skin candidate list: every (j, image) within r_nb + skin at the last build
struct CandList {
  int cap;
  int* cnt;
  int* j;
  uint8_t* s;
  float rc2;                   // (r_nb + skin)^2 plus a rounding margin
  double half_skin2;           // (skin / 2)^2: rebuild when an atom moved farther
};

struct Cells {
  const int* nc;               // [nrep*3]
  const int* cell_off;         // [nrep+1] first cell of each replica
  int ncell_total;
  int* count;                  // [ncell_total]
  int* start;                  // [ncell_total+1]
  int* cursor;                 // [ncell_total]
  int* atoms;                  // [n] atoms sorted by cell
  int* atom_cell;              // [n]
  int* tmp;                    // [n] scatter scratch
  int slices;                  // blocks per home cell in the candidate build (>= 1)
};

// Far list. Context path: every row is split into a near part (r < r_bond, the bond
// candidates; capn, cntn, jn, sn, Hn) and a far part (r_bond <= r < r_nb; cap, cnt, j, s,
// H). The allocation-free builder fills only the single (unsplit) part.
struct FarList {
  int cap;
  int* cnt;                    // [n]
  int* j;                      // [n*cap]
  uint8_t* s;                  // [n*cap]
  void* H;                     // [n*cap] of R: QEq matrix off-diagonal entries
  int capn;
  int* cntn;
  int* jn;
  uint8_t* sn;
  void* Hn;
  double r2_nb, r2_bond, r2_hb; // squared cutoffs (precomputed on the host)
};

struct BondList {
  int cap;
  int* cnt;
  int* j;
  uint8_t* s;
  int* mirror;                 // global entry index of the reverse entry
  int* canon;                  // compact list of canonical entries (one per unordered bond)
  int* ncanon;                 // its length (device counter)
  // geometry (arrays of R, [n*cap])
  void *dx, *dy, *dz, *r;
  // BO' (shifted total), pi, pipi and their r-derivatives: FP64 in both modes, because the
  // correction f1 depends on Delta' = sum BO' - Val through e^{-p_boc1 Delta'} (p_boc1 ~ 50)
  double *bop, *bopi, *bopp, *dbop, *dbopi, *dbopp;
  void *bo, *bo_pi, *bo_pp;                            // corrected
  void *f1, *fo, *ft, *df1, *dfo_bo, *dft_bo, *dfo_d;  // correction factors and partials
  double *dEdBOp, *dEdBOpi, *dEdBOpp;                  // chain-rule coefficients
  unsigned long long *cdbo, *cdbopi, *cdbopp;          // dE/dBO accumulators (fixed point)
};

struct HbList {
  int cap;
  int* cnt;
  int* j;
  uint8_t* s;
};

struct AtomQ {                 // per-atom bond-order quantities (double)
  double *dp, *dpboc;          // Delta', Delta'boc
  double *sumbo, *delta, *dang, *nlp, *dnlp, *dlp, *dd;   // dd = Delta - Delta_lp
  double *prodexp, *sbo2, *dsbo2, *sbo_fac;               // sbo_fac = -Delta_ang - p_val8 nlp
  double* cds;                 // dE/dS
  unsigned long long* A;       // chain-rule dE/dDelta' per atom (fixed point)
  unsigned long long* cddelta; // dE/d(sum BO) accumulator (fixed point)
  float *sumbo_f, *dang_f;     // FP32 copies for the mixed-path angle and torsion kernels
  float *delta_f, *sbo2_f, *dsbo2_f, *prodexp_f, *sbo_fac_f, *dnlp_f;
};

struct Accum {                 // per-atom energies and virial
  double* e;                   // [NTERMS*n] owner-written
  double* vir;                 // [6*n] owner-accumulated
  unsigned long long* efx;     // [NTERMS*n] energies added as 2^-32 fixed point (atomics, or FP32
                               // warp totals without FP64 conversions), per term like e
  unsigned long long* vfx;     // [6*n] virial contributions added by atomics (fixed point)
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ long long fix_of(double v, int* err) {
  if (!(fabs(v) < FIX_LIMIT)) {
    atomicOr(err, ERR_NAN);
    return 0;
  }
  return __double2ll_rn(v * FIX_SCALE);
}
__device__ __forceinline__ void fix_add(unsigned long long* p, double v, int* err) {
  long long f = fix_of(v, err);
  if (f != 0) atomicAdd(p, (unsigned long long)f);
}
// FP32 value -> 2^32 fixed point with 32-bit conversions only (GB300 issues 64-bit
// conversions at the FP64 rate, ~16x slower than 32-bit ones). t = v 2^32 is exact; for
// |t| < 2^31 a 32-bit round-to-nearest conversion gives round(t); a larger |t| is already
// an integer (its ulp is >= 2^8) and is rebuilt exactly from its bits. The result equals
// what a 64-bit round-to-nearest conversion of t gives.
__device__ __forceinline__ long long fix_of_f(float v) {
  const float t = v * 4294967296.0f;
  if (fabsf(t) < 2147483648.0f) return (long long)__float2int_rn(t);
  const int b = __float_as_int(t);
  const int e = ((b >> 23) & 0xff) - 150;           // t = m 2^e, 8 <= e <= 38 below FIX_LIMIT
  const long long mag = (long long)((b & 0x7fffff) | 0x800000) << e;
  return b < 0 ? -mag : mag;
}
__device__ __forceinline__ void fix_add(unsigned long long* p, float v, int* err) {
  if (!(fabsf(v) < (float)FIX_LIMIT)) {
    atomicOr(err, ERR_NAN);
    return;
  }
  const long long f = fix_of_f(v);
  if (f != 0) atomicAdd(p, (unsigned long long)f);
}
// a float-float value hi + lo (|lo| <= ulp(hi)/2): both parts converted, then summed
__device__ __forceinline__ void fix_add_ff(unsigned long long* p, float hi, float lo, int* err) {
  if (!(fabsf(hi) < (float)FIX_LIMIT)) {
    atomicOr(err, ERR_NAN);
    return;
  }
  const long long f = fix_of_f(hi) + fix_of_f(lo);
  if (f != 0) atomicAdd(p, (unsigned long long)f);
}
__device__ __forceinline__ double fix_get(const unsigned long long* p) {
  return (double)(long long)(*p) * FIX_INV;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Deterministic warp sum of FP32 lane partials in float-float (TwoSum) arithmetic: only
// FP32 instructions (GB300 runs FP64 at 1/64 of the FP32 rate, and an FP64 butterfly
// costs 5 FP64 adds in every lane); exact to ~2^-48 of the partials. The same value
// in every lane (the error term of a TwoSum is unique, so the butterfly is symmetric).
// error-free sum: s + e == a + b exactly (Knuth TwoSum, FP32)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// float-float butterfly: on return every lane holds the warp total of the (hi, lo) pairs
__device__ __forceinline__ void warp_sum_ff2(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ohi, s, e);
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
    hi = s;
  }
}
__device__ __forceinline__ double warp_sum_ff(float v) {
  float hi = v, lo = 0.0f;
  warp_sum_ff2(hi, lo);
  return (double)hi + (double)lo;
}
// lane q takes value q of N float-float totals held by every lane (q >= N: zeros). Used
// to spread the few FP64 conversions of a warp's results over its lanes, so that one
// warp instruction converts them all.
template <int N>
__device__ __forceinline__ void lane_pick(const float* hi, const float* lo, int q, float& h, float& l) {
  h = 0.0f;
  l = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k == q) {
      h = hi[k];
      l = lo[k];
    }
}
__device__ __forceinline__ double warp_sum_d(float v) { return warp_sum_ff(v); }
__device__ __forceinline__ double warp_sum_d(double v) { return warp_sum(v); }
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void shift_decode(int code, int& sx, int& sy, int& sz) {
  sx = code / 9 - 1;
  sy = (code / 3) % 3 - 1;
  sz = code % 3 - 1;
}

// precision-generic math wrappers
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float m_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float m_cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double m_acos(double x) { return acos(x); }
__device__ __forceinline__ float m_acos(float x) { return acosf(x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
// MUFU-based fast variants (FP32) for far pairs whose contributions are small; the
// FP64 path keeps the accurate functions
__device__ __forceinline__ double f_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float f_pow(float x, float y) { return __powf(x, y); }
__device__ __forceinline__ double f_exp(double x) { return exp(x); }
__device__ __forceinline__ float f_exp(float x) { return __expf(x); }
// exp with the argument capped so FP32 never overflows to inf (inf*0 -> NaN in the
// derivative products); the cap is far beyond any value that changes an FP64 result
template <typename R> __device__ __forceinline__ R exp_cap_arg();
template <> __device__ __forceinline__ double exp_cap_arg<double>() { return 700.0; }
template <> __device__ __forceinline__ float exp_cap_arg<float>() { return 80.0f; }
template <typename R> __device__ __forceinline__ R m_expc(R x) {
  return m_exp(x < exp_cap_arg<R>() ? x : exp_cap_arg<R>());
}
template <typename R> __device__ __forceinline__ R rclamp(R x, R lo, R hi) {
  return x < lo ? lo : (x > hi ? hi : x);
}
// 1 / (1 + exp(u)) and its derivative -s(1-s), overflow-safe
template <typename R> __device__ __forceinline__ R sig_neg(R u) {
  return R(1) / (R(1) + m_expc(u));
}
// s = 1/(1 + e^u) and sd = s (1 - s) = e^u s^2 without the cancellation of 1 - s
template <typename R> __device__ __forceinline__ void sig_pair(R u, R& s, R& sd) {
  const R e = m_expc(u);
  s = R(1) / (R(1) + e);
  sd = e * s * s;
}
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
// a*b - c*d with one rounding error (fma-based; Kahan's difference of products)
__device__ __forceinline__ double diff_prod(double a, double b, double c, double d) { return a * b - c * d; }
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = __fmaf_rn(-c, d, w);
  const float f = __fmaf_rn(a, b, -w);
  return f + e;
}
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }

// taper Tap(x) = 20x^7 - 70x^6 + 84x^5 - 35x^4 + 1 and dTap/dr, x = r/R
template <typename R> __device__ __forceinline__ void taper(R r, R Rc, R& t, R& dt) {
  R x = r / Rc;
  R x2 = x * x, x3 = x2 * x;
  t = ((((R(20) * x - R(70)) * x + R(84)) * x - R(35)) * x2 * x2) + R(1);
  dt = ((((R(140) * x - R(420)) * x + R(420)) * x - R(140)) * x3) / Rc;
}

// Image vector d = (x_j - x_i) + s*L of a list entry (shift code 0..26).
// FP64: the defining arithmetic. FP32: hi/lo float positions with an error-free
// difference of the hi parts, so d is within ~1 ulp of its own magnitude (not of L).
template <typename R> struct PairVec;
template <> struct PairVec<double> {
  static __device__ __forceinline__ void get(const Sys& s, int i, int j, int code, int r, double& dx,
                                             double& dy, double& dz) {
    int sx, sy, sz;
    shift_decode(code, sx, sy, sz);
    const double* L = s.box + 3 * r;
    dx = __dadd_rn(__dsub_rn(s.x[j], s.x[i]), sx == 0 ? 0.0 : (sx > 0 ? L[0] : -L[0]));
    dy = __dadd_rn(__dsub_rn(s.y[j], s.y[i]), sy == 0 ? 0.0 : (sy > 0 ? L[1] : -L[1]));
    dz = __dadd_rn(__dsub_rn(s.z[j], s.z[i]), sz == 0 ? 0.0 : (sz > 0 ? L[2] : -L[2]));
  }
};
__device__ __forceinline__ float pv_comp(float hj, float hi, float lj, float li, int sgn, float Lh,
                                         float Ll) {
  float d, e;
  two_sum(hj, -hi, d, e);
  float a = sgn == 0 ? d : __fadd_rn(d, sgn > 0 ? Lh : -Lh);
  float t = __fadd_rn(__fadd_rn(e, __fsub_rn(lj, li)), sgn == 0 ? 0.0f : (sgn > 0 ? Ll : -Ll));
  return __fadd_rn(a, t);
}
// float-float image vector: d = dh + dl with |dl| <= ulp(dh)/2 (error-free transforms)
__device__ __forceinline__ void pv_comp_ff(float hj, float hi, float lj, float li, int sgn, float Lh, float Ll,
                                           float& dh, float& dl) {
  float d, e;
  two_sum(hj, -hi, d, e);
  float a, e2;
  if (sgn == 0) { a = d; e2 = 0.0f; }
  else two_sum(d, sgn > 0 ? Lh : -Lh, a, e2);
  const float t = __fadd_rn(__fadd_rn(__fadd_rn(e, e2), __fsub_rn(lj, li)), sgn == 0 ? 0.0f : (sgn > 0 ? Ll : -Ll));
  two_sum(a, t, dh, dl);
}
// float-float |d|: r = rh + rl from exact squares (fma) and one Newton correction
__device__ __forceinline__ void norm_ff(const float* dh, const float* dl, float& rh, float& rl) {
  float sh = 0.0f, sl = 0.0f;
  for (int c = 0; c < 3; ++c) {
    const float p = __fmul_rn(dh[c], dh[c]);
    const float pe = __fmaf_rn(dh[c], dh[c], -p);
    float t, te;
    two_sum(sh, p, t, te);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, __fadd_rn(pe, 2.0f * dh[c] * dl[c])));
  }
  float s, se;
  two_sum(sh, sl, s, se);
  rh = sqrtf(s);
  const float q = __fmul_rn(rh, rh);
  const float qe = __fmaf_rn(rh, rh, -q);
  rl = (((s - q) - qe) + se) / (2.0f * rh);
}

template <> struct PairVec<float> {
  // image vector from the packed records (two 16-byte gathers per atom); hj, lj return
  // atom j's records for the caller's use of the charge and type fields
  static __device__ __forceinline__ void getv(const Sys& s, int i, int j, int code, int r, float& dx, float& dy,
                                              float& dz, float4& hj, float4& lj) {
    int sx, sy, sz;
    shift_decode(code, sx, sy, sz);
    const float* Lh = s.boxh + 3 * r;
    const float* Ll = s.boxl + 3 * r;
    hj = s.ph[j];
    lj = s.pl[j];
    const float4 hi = s.ph[i], li = s.pl[i];
    dx = pv_comp(hj.x, hi.x, lj.x, li.x, sx, Lh[0], Ll[0]);
    dy = pv_comp(hj.y, hi.y, lj.y, li.y, sy, Lh[1], Ll[1]);
    dz = pv_comp(hj.z, hi.z, lj.z, li.z, sz, Lh[2], Ll[2]);
  }
  static __device__ __forceinline__ void get(const Sys& s, int i, int j, int code, int r, float& dx,
                                             float& dy, float& dz) {
    float4 hj, lj;
    getv(s, i, j, code, r, dx, dy, dz, hj, lj);
  }
};
// Fourth word of a pl record: type (8 bits) and the three box-crossing counters since the
// last candidate-list build (8-bit two's complement each; an atom moves less than half the
// skin between builds, so each counter is -1, 0 or 1 there)
__device__ __forceinline__ float pack_type_img(int type, int ix, int iy, int iz) {
  return __int_as_float((type & 0xff) | ((ix & 0xff) << 8) | ((iy & 0xff) << 16) | ((iz & 0xff) << 24));
}
__device__ __forceinline__ int rec_type(float w) { return __float_as_int(w) & 0xff; }
__device__ __forceinline__ void rec_img(float w, int& ix, int& iy, int& iz) {
  const int b = __float_as_int(w);
  ix = (b << 16) >> 24;
  iy = (b << 8) >> 24;
  iz = b >> 24;
}
// FP32 hi/lo position copies of atom i: the split arrays and, when present, the packed
// records (the charge field is left to the charge writers)
__device__ __forceinline__ void write_pos_f32(const Sys& s, int i) {
  const float xh = (float)s.x[i], yh = (float)s.y[i], zh = (float)s.z[i];
  const float xl = (float)(s.x[i] - (double)xh), yl = (float)(s.y[i] - (double)yh), zl = (float)(s.z[i] - (double)zh);
  s.xh[i] = xh; s.yh[i] = yh; s.zh[i] = zh;
  s.xl[i] = xl; s.yl[i] = yl; s.zl[i] = zl;
  if (s.ph) {
    float* h = (float*)(s.ph + i);
    h[0] = xh; h[1] = yh; h[2] = zh;
    s.pl[i] = make_float4(xl, yl, zl, pack_type_img(s.type[i], s.img[3 * i], s.img[3 * i + 1], s.img[3 * i + 2]));
  }
}
__device__ __forceinline__ void write_q_f32(const Sys& s, int i, double q) {
  const float qf = (float)q;
  s.qf[i] = qf;
  if (s.ph) ((float*)(s.ph + i))[3] = qf;
}
// r^2 exactly as the list definition fixes it (FP64, no contraction)
__device__ __forceinline__ double r2_exact(const Sys& s, int i, int j, int code, int r) {
  double dx, dy, dz;
  PairVec<double>::get(s, i, j, code, r, dx, dy, dz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ------------------------------------------------------------------ bounded grid barrier
// Used only inside cooperative launches (all blocks co-resident). Sense via a
// generation counter; gives up after `limit` polls, sets ERR_TIMEOUT and returns false.
struct GridBar {
  unsigned int arrive;
  unsigned int gen;
};
constexpr long long BAR_SPIN_LIMIT = 20000000LL;    // ~1-2 s of polling (64 ns sleeps)
constexpr long long BAR_CYCLE_LIMIT = 3000000000LL; // ~1.5 s of SM clock at 2 GHz

// ------------------------------------------------------------------ host side
struct reaxff_ctx_impl;
std::string cuda_err_str(cudaError_t e);

// kernel entry points (host launch wrappers), defined in the .cu files
namespace rx {
// launch schedules picked by the autotuner (reaxff_autotune); defaults otherwise
struct Tune {
  int tors_lanes = 4;          // lanes per central bond in the torsion kernel (1 mixed path only, 2, 4, 8)
  int nb_block = 256;          // threads per block: nonbonded (warp per atom)
  int cf_block = 256;          //   candidate filter (warp per atom)
  int bl_block = 256;          //   bond list (warp per atom)
  int ang_block = 128;         //   angles
  int ang_lanes = 8;           // lanes per centre atom in the angle kernel (4, 8, 16, 32; mixed path)
  int hb_block = 128;          //   H-bonds (warp per hydrogen)
  int qeq_overlap = 0;         // 1 / 2: QEq (CG on 512 / 256 threads per SM) runs beside the
                               //    charge-free bond-order and bonded kernels (mixed path);
                               //    3..5: beside them on 1024-thread blocks, launch shape
                               //    qeq_overlap - 2
};
struct Launch {
  cudaStream_t st;
  int64_t* count;              // launch counter
  const Tune* tune = nullptr;  // schedules (null: defaults)
  const Tune& t() const {
    static const Tune def{};
    return tune ? *tune : def;
  }
};
// lists.cu
void cells_build(const Launch& L, Sys s, Cells c);
template <typename R>
void far_list(const Launch& L, Sys s, Cells c, FarList f, const DParams<R>* P, float margin);
template <typename R>
void far_list_split(const Launch& L, Sys s, Cells c, FarList f, const DParams<R>* P, float margin,
                    float margin_near);
void charges_to_f32(const Launch& L, Sys s);
// skin list: float position copies (every step), displacement check, conditional cell
// binning + candidate build, exact per-step filter into the near/far rows
void positions_f32(const Launch& L, Sys s);
void skin_check(const Launch& L, Sys s, CandList cl);
void cand_build(const Launch& L, Sys s, Cells c, CandList cl);
template <typename R>
void cand_filter(const Launch& L, Sys s, CandList cl, FarList f, HbList h, const DParams<R>* P, float margin,
                 float margin_near, float margin_hb);
template <typename R>
void bond_list(const Launch& L, Sys s, FarList f, BondList b, HbList h, AtomQ a, const DParams<R>* P,
               const DParams<double>* Pd, bool hb_built = false);   // hb_built: cand_filter made the H-bond list
void bond_mirror(const Launch& L, Sys s, BondList b);
void bo_prime64(const Launch& L, Sys s, BondList b, AtomQ a, const DParams<double>* Pd, int n_canon_max);
// bonded.cu
template <typename R>
void bo_correct(const Launch& L, Sys s, BondList b, AtomQ a, const DParams<R>* P);
template <typename R>
void atom_terms(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P,
                unsigned mask);
template <typename R>
void over_under_bond(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P,
                     unsigned mask);
template <typename R>
void s_gather(const Launch& L, Sys s, BondList b, AtomQ a);
template <typename R>
void angles(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P, unsigned mask);
template <typename R>
void torsions(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc, const DParams<R>* P,
              unsigned mask);
template <typename R>
void hbonds(const Launch& L, Sys s, BondList b, HbList h, Accum acc, const DParams<R>* P,
            unsigned mask);
// nonbonded.cu
template <typename R>
void nonbonded(const Launch& L, Sys s, FarList f, Accum acc, const DParams<R>* P, unsigned mask);
// forces.cu
template <typename R>
void chain_rule(const Launch& L, Sys s, BondList b, AtomQ a, Accum acc);
void finalize_forces(const Launch& L, Sys s, double* F);
constexpr int RED_CHUNK = 512;   // atoms per reduction chunk
struct RedPlan {                // chunks (<= RED_CHUNK atoms, never straddling replicas) for reductions
  int nchunk;
  int* chunk_lo;               // [nchunk+1]
  int* chunk_rep;              // [nchunk] replica of each chunk
  int* rep_chunk;              // [nrep+1]
  double* part;                // [nchunk*20]
  unsigned* done;              // arrival counters [nrep*20 + nrep + 1] (zero between launches)
};
// per-replica energies, virial and kinetic energy; with etot, also the total energy per
// replica into etot[k*nrep + r], k = *etot_idx (then advanced) or 0 without etot_idx
void reduce_energies(const Launch& L, Sys s, Accum acc, const double* mass_t, const RedPlan& rp, double* E_rep,
                     double* vir_rep, double* ke_rep, double* etot = nullptr, int* etot_idx = nullptr);
void verlet_kick_drift(const Launch& L, Sys s, const double* mass_t, double dt, int drift,
                       const CandList* cl = nullptr);   // cl: also float records + skin test
// save (restore = 0) or restore the primary MD state: x, v, the QEq rings (contiguous,
// nhist_doubles) and their device state hst[4]; buf holds 6n + nhist_doubles doubles
void snapshot(const Launch& L, Sys s, double* hist, int nhist_doubles, int* hst, double* buf, int* ibuf, int restore);
// qeq.cu
// QEq solver state. The cooperative kernel keeps each block's per-replica scalars and the
// CG vectors of its rows in dynamic shared memory when they fit in QEQ_SMEM_MAX bytes,
// else in block-private global regions (scal, state).
constexpr int QEQ_SMEM_MAX = 200 * 1024;
constexpr int QEQ_NV_STATE = 14;             // doubles per row of CG state
constexpr int QEQ_HIST = 8;                  // solutions kept per system for the initial guess
constexpr int QEQ_NPRED = 3;                 // initial-guess predictors: Lagrange, least squares over 6, over 8
constexpr int QEQ_SCAL_PER_REP = 24;         // doubles per replica of scalars + reductions
// One cooperative launch shape of the solve: the grid, the chunks of rows (runs of atoms of
// one replica; block b owns chunks b, b + grid, ...) and where each block keeps its row state,
// scalars and block inverses. Shape 0 has one block on every SM (1024, 512 or 256 threads);
// the others have 1024-thread blocks on a part of the SMs, which leaves the rest of the GPU
// whole to the kernels running beside the solve.
struct QeqLayout {
  int grid;                    // blocks
  int nchunk;
  int* chunk_lo;               // first atom of each chunk [nchunk+1]
  int* chunk_rep;              // replica of each chunk
  int* rep_chunk;              // first chunk of each replica [nrep+1]
  int rows_blk;                // most rows one block owns
  int scal_smem, state_smem;   // 1: held in dynamic shared memory
  int bj_smem;                 // 1: each block's inverses staged in its shared memory
  int smem_bytes;              // dynamic shared memory of the launch
};
// shapes 1.. : grid = QEQ_PART_NUM[k] / 8 of the SMs
constexpr int QEQ_NLAYOUT = 4;
constexpr int QEQ_PLACEMENTS = 2 + QEQ_NLAYOUT;   // schedule entry qeq_overlap: 0 .. QEQ_PLACEMENTS - 1
constexpr int QEQ_PART_NUM[QEQ_NLAYOUT] = {8, 4, 3, 5};
struct QeqState {
  double *hist_s, *hist_t;     // [QEQ_HIST*n] each: solution rings (s, t); the solver writes
                               // each new solution into the oldest slot
  double* wext;                // [QEQ_NPRED][2][QEQ_HIST+1][QEQ_HIST] guess weights by history length
  int* pred;                   // [2*nrep] predictor in use per replica and system (s, t)
  int* hst;                    // device {slot of the newest s, of the newest t, usable entries}
  void* zg;                    // interleaved (s, t) copy of the SpMV operand: float2 or double2
  const double* ieta;          // 1/eta per type
  double* part;                // chunk partials [2][8][nchunk] (the most chunks of any shape)
  double* scal;                // [grid][nrep*24+4] per-block scalars (when not in shared memory)
  double* state;               // [grid][14][rows_blk] per-block row state (when not in shared memory)
  int ring_bytes;              // SpMV streaming ring (mixed path; first in the shared memory layout)
  QeqLayout lay[QEQ_NLAYOUT];  // launch shapes
  int* iters;                  // [2*nrep]
  unsigned long long* spmv_total;   // SpMVs of all solves since creation
  int* mlp_used;               // [nrep] learned guess kept in the last solve
  GridBar* bar;
  // block-Jacobi preconditioner (REAXFF_PRECOND_BLOCK32): blocks of 32 consecutive atoms of a
  // replica; element (t, m) of the symmetrised FP32 inverse of the block starting at atom b0
  // at binv[32 (b0 + m) + t] (32 (n + 32) floats); null for Jacobi
  int precond;
  float* binv;
  int* bj_start;               // [bj_nblk] first atom of each block
  int* bj_size;                // [bj_nblk] atoms in the block (32, fewer at a replica's end)
  int bj_nblk;
  const DParams<float>* Pf;    // FP32 parameters for the block build
  long long bar_limit;         // grid-barrier wait limit in SM cycles (0: BAR_CYCLE_LIMIT)
};
// qhat (device, or null): learned charges offered as a second starting guess for s
template <typename R>
int qeq_solve(const Launch& L, Sys s, FarList f, QeqState& Q, const DParams<R>* P, const double* chi,
              const double* eta, double tol, int max_iter, int warm, const float* qhat, int threads = 1024,
              int layout = 0);
int qeq_grid_size(int nsm);
int qeq_ring_bytes(bool fp64);   // shared memory of the SpMV streaming ring of a 1024-thread block
void qeq_precond_build(const Launch& L, Sys s, QeqState& Q);   // block-Jacobi inverses (no-op for Jacobi)

// mlp.cu: learned QEq warm start (descriptors, BF16 tensor-core inference, FP32 training)
constexpr int MLP_NF = 192, MLP_HID = 64, MLP_NT = 4;
constexpr int MLP_NPAR = MLP_NF * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID + 1;   // per element
struct MlpScratch {            // per-sample training activations and gradients
  float *z1, *z2, *dz1, *dz2;  // [m][64]
  float *y, *l;                // [m]
  float* part;                 // [ceil(m / 256)][4 * 16577] weight-gradient chunk partials
};
constexpr int MLP_WG_CHUNK = 256;
struct MlpTiles {              // tiles of <= 128 rows of one element, rows in element order
  int rows, ntile;
  int* perm;                   // [rows] packed row -> sample
  int* tile_type;              // [ntile]
  int* rows_off;               // [ntile + 1]
};
struct MlpInfer {              // BF16 operands of the tensor-core forward
  void* Xp;                    // [rows][192] BF16 normalised inputs
  void* W1t;                   // [4][64][192] BF16
  void* W2t;                   // [4][64][64] BF16
  float* fp;                   // [4][193] b1, b2, w3, b3
};
// gate (device QEq history state, or null): skip the work when a solution history exists
void mlp_descriptors(const Launch& L, Sys s, FarList f, float* D, const int* gate = nullptr);
void mlp_stats(const Launch& L, const float* X, int64_t rows, float* mean, float* inv);
void mlp_loss_grad(const Launch& L, const float* X, const int* type, const int* idx, const int* off, const float* Q,
                   int m, const float* theta, const float* mean, const float* inv, MlpScratch& w, float* G,
                   double* loss);
void mlp_forward32(const Launch& L, const float* X, const int* type, int m, const float* theta, const float* mean,
                   const float* inv, MlpScratch& w);
void mlp_adam(const Launch& L, float* theta, const float* g, float* mo, float* vo, int step, float lr);
// BF16 tensor-core operands from the FP32 parameters (after every parameter change)
void mlp_weights(const Launch& L, const float* theta, MlpInfer& w);
// y[perm-order samples] = network(D) on the tensor cores (uses the converted weights)
void mlp_infer(const Launch& L, const float* D, const MlpTiles& T, const float* mean, const float* inv,
               MlpInfer& w, float* y_out, int* err, int nsm, const int* gate = nullptr);
int mlp_tc_setup();

// species.cu: molecular species analysis
struct SpeciesBuf {
  int *lab, *rank, *mol;       // [n] root labels, root ranks, molecule of each atom
  int *cnt, *mrep;             // [n*MAXT] element counts per molecule, [n] replica per molecule
  int *boff, *nmol, *changed;  // block offsets, molecule count, hook flag
  int* h_changed;              // pinned host copy of the flag
};
template <typename R>
int species_components(const Launch& L, Sys s, BondList bl, const double* thr, SpeciesBuf& b, int max_pass);
void species_molecules(const Launch& L, Sys s, SpeciesBuf& b);
// time-averaged bond orders: per atom a row of cap (j, image code, running sum) entries keyed
// by the neighbour and its image; avg = sum / samples is written by bo_average_finish
struct BoAvg {
  int cap;
  int* cnt;                    // [n] entries in use
  int* j;                      // [n*cap]
  uint8_t* s;                  // [n*cap] image code
  double *sum, *avg;           // [n*cap]
  int* over;                   // set when a row had no room for a new pair
};
template <typename R>
void bo_average_sample(const Launch& L, Sys s, BondList bl, BoAvg A);
void bo_average_finish(const Launch& L, int n, BoAvg A, double inv_samples);
}  // namespace rx

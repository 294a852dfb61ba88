// (a) Cell binning, far-neighbour list (+ QEq H entries), bond list (+ BO'), H-bond list.
//
// Paper: Sec. 3.3 "Neighbor and Interaction Lists" (own far list with distances, compact
// adjacency rows, bond and H-bond lists generated from one pass over the neighbour
// list) and Sec. 3.2 (spatial order of atoms). GPU form: the cell grid is binned with a
// count -> scan -> scatter and a per-cell rank sort (deterministic order, no slot locks);
// one warp builds one atom's row: 27 stencil cells with image shifts, 32 candidates per
// ballot, warp-compacted writes. Membership is decided exactly as the FP64 definition
// (d = (xj - xi) + s*L, r^2 = (dx*dx + dy*dy) + dz*dz, r^2 < R^2) using an FP32 filter
// with a proven error margin and FP64 only inside the margin.
#include "reax_internal.cuh"

namespace {

template <bool COND>
__global__ void k_cell_assign(Sys s, Cells c) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  if (COND && *s.rebuild == 0) return;
  int r = s.rep[i];
  const double* L = s.box + 3 * r;
  const int* nc = c.nc + 3 * r;
  double p[3] = {s.x[i], s.y[i], s.z[i]};
  int cc[3];
  for (int d = 0; d < 3; ++d) {
    int k = (int)floor(p[d] / L[d] * (double)nc[d]);
    cc[d] = k < 0 ? 0 : (k >= nc[d] ? nc[d] - 1 : k);
  }
  int cell = c.cell_off[r] + (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
  c.atom_cell[i] = cell;
  atomicAdd(&c.count[cell], 1);
  write_pos_f32(s, i);   // float hi/lo copies of the positions
}

// single-block exclusive scan over cell counts
template <bool COND>
__global__ void k_cell_scan(Cells c, const int* rebuild) {
  if (COND && *rebuild == 0) return;
  __shared__ int carry;
  __shared__ int warp_tot[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < c.ncell_total; base += blockDim.x) {
    int k = base + threadIdx.x;
    int v = k < c.ncell_total ? c.count[k] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      int nw = blockDim.x >> 5;
      int t = lane < nw ? warp_tot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      if (lane < nw) warp_tot[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    int excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + incl - v;
    if (k < c.ncell_total) {
      c.start[k] = excl;
      c.cursor[k] = excl;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) c.start[c.ncell_total] = carry;
}

template <bool COND>
__global__ void k_cell_scatter(Sys s, Cells c, int* tmp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  if (COND && *s.rebuild == 0) return;
  int slot = atomicAdd(&c.cursor[c.atom_cell[i]], 1);
  tmp[slot] = i;
}

// per cell: order atoms by index (rank = number of smaller indices in the cell)
template <bool COND>
__global__ void k_cell_sort(Cells c, const int* tmp, const int* rebuild) {
  if (COND && *rebuild == 0) return;
  int cell = blockIdx.x;
  int a = c.start[cell], b = c.start[cell + 1];
  for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
    int me = tmp[k];
    int rank = 0;
    for (int m = a; m < b; ++m) rank += tmp[m] < me;
    c.atoms[a + rank] = me;
  }
}

// decide r^2 < R2 exactly (FP64 definition) from an FP32 estimate with error bound `margin`
__device__ __forceinline__ bool in_range(const Sys& s, int i, int j, int code, int r, float r2f, float R2f,
                                         float margin, double R2) {
  if (r2f < R2f - margin) return true;
  if (r2f > R2f + margin) return false;
  return r2_exact(s, i, j, code, r) < R2;
}

template <typename R>
__global__ void k_far_list(Sys s, Cells c, FarList f, const DParams<R>* __restrict__ P, float margin) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= s.n) return;
  const int i = warp;
  const int r = s.rep[i];
  const int* nc = c.nc + 3 * r;
  const float* Lh = s.boxh + 3 * r;
  const double Rc = (double)P->r_nb;
  const double R2 = Rc * Rc;
  const float R2f = (float)R2;
  int cell = c.atom_cell[i] - c.cell_off[r];
  int ci[3] = {cell % nc[0], (cell / nc[0]) % nc[1], cell / (nc[0] * nc[1])};
  float xi = s.xh[i], yi = s.yh[i], zi = s.zh[i];
  const int ti = s.type[i];
  int count = 0;
  const int base_row = i * f.cap;
  R* H = (R*)f.H;
  for (int o = 0; o < 27; ++o) {
    int oc[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    int t[3], sh[3];
    for (int d = 0; d < 3; ++d) {
      int v = ci[d] + oc[d];
      sh[d] = v < 0 ? -1 : (v >= nc[d] ? 1 : 0);
      t[d] = v - sh[d] * nc[d];
    }
    int code = (sh[0] + 1) * 9 + (sh[1] + 1) * 3 + (sh[2] + 1);
    int cid = c.cell_off[r] + (t[2] * nc[1] + t[1]) * nc[0] + t[0];
    int a = c.start[cid], b = c.start[cid + 1];
    float ox = sh[0] * Lh[0], oy = sh[1] * Lh[1], oz = sh[2] * Lh[2];
    for (int base = a; base < b; base += 32) {
      int k = base + lane;
      bool ok = false;
      int j = -1;
      if (k < b) {
        j = c.atoms[k];
        float dx = (s.xh[j] - xi) + ox, dy = (s.yh[j] - yi) + oy, dz = (s.zh[j] - zi) + oz;
        float r2f = dx * dx + dy * dy + dz * dz;
        ok = !(j == i && code == 13) && in_range(s, i, j, code, r, r2f, R2f, margin, R2);
      }
      unsigned m = __ballot_sync(0xffffffffu, ok);
      int pos = count + __popc(m & ((1u << lane) - 1u));
      if (ok && pos < f.cap) {
        f.j[base_row + pos] = j;
        f.s[base_row + pos] = (uint8_t)code;
        R dx, dy, dz;
        PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
        R rr = m_sqrt(dx * dx + dy * dy + dz * dz);
        R tap, dtap;
        taper<R>(rr, P->r_nb, tap, dtap);
        R g3 = P->gamma_m3[ti * MAXT + s.type[j]];
        H[base_row + pos] = tap * P->k_e / m_cbrt(rr * rr * rr + g3);
      }
      count += __popc(m);
    }
  }
  if (lane == 0) {
    f.cnt[i] = count < f.cap ? count : f.cap;
    if (count > f.cap) atomicOr(s.err, ERR_CAP_FAR);
  }
}

// Context-path far list: the same candidates and exact membership as k_far_list, each
// accepted entry written to the near part (r < r_bond, exact FP64 decision in the band)
// or the far part of its row.
template <typename R>
__global__ void k_far_list_split(Sys s, Cells c, FarList f, const DParams<R>* __restrict__ P, float margin,
                                 float margin_near, double R2, double Rb2) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= s.n) return;
  const int i = warp;
  const int r = s.rep[i];
  const int* nc = c.nc + 3 * r;
  const float* Lh = s.boxh + 3 * r;
  const float R2f = (float)R2;        // R2, Rb2 come precomputed (no FP64 work in the loop)
  const float Rb2f = (float)Rb2;
  int cell = c.atom_cell[i] - c.cell_off[r];
  int ci[3] = {cell % nc[0], (cell / nc[0]) % nc[1], cell / (nc[0] * nc[1])};
  float xi = s.xh[i], yi = s.yh[i], zi = s.zh[i];
  const int ti = s.type[i];
  int cntn = 0, cntf = 0;
  const int rown = i * f.capn, rowf = i * f.cap;
  R* Hn = (R*)f.Hn;
  R* Hf = (R*)f.H;
  for (int o = 0; o < 27; ++o) {
    int oc[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    int t[3], sh[3];
    for (int d = 0; d < 3; ++d) {
      int v = ci[d] + oc[d];
      sh[d] = v < 0 ? -1 : (v >= nc[d] ? 1 : 0);
      t[d] = v - sh[d] * nc[d];
    }
    int code = (sh[0] + 1) * 9 + (sh[1] + 1) * 3 + (sh[2] + 1);
    int cid = c.cell_off[r] + (t[2] * nc[1] + t[1]) * nc[0] + t[0];
    int a = c.start[cid], b = c.start[cid + 1];
    float ox = sh[0] * Lh[0], oy = sh[1] * Lh[1], oz = sh[2] * Lh[2];
    for (int base = a; base < b; base += 32) {
      int k = base + lane;
      bool ok = false, near = false;
      int j = -1;
      if (k < b) {
        j = c.atoms[k];
        float dx = (s.xh[j] - xi) + ox, dy = (s.yh[j] - yi) + oy, dz = (s.zh[j] - zi) + oz;
        float r2f = dx * dx + dy * dy + dz * dz;
        ok = !(j == i && code == 13) && in_range(s, i, j, code, r, r2f, R2f, margin, R2);
        if (ok) near = in_range(s, i, j, code, r, r2f, Rb2f, margin_near, Rb2);
      }
      const unsigned mn = __ballot_sync(0xffffffffu, ok && near);
      const unsigned mf = __ballot_sync(0xffffffffu, ok && !near);
      const unsigned below = (1u << lane) - 1u;
      if (ok) {
        R dx, dy, dz;
        PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
        const R rr = m_sqrt(dx * dx + dy * dy + dz * dz);
        R tap, dtap;
        taper<R>(rr, P->r_nb, tap, dtap);
        const R g3 = P->gamma_m3[ti * MAXT + s.type[j]];
        const R sh3 = rr * rr * rr + g3;
        if (near) {
          const int pos = cntn + __popc(mn & below);
          if (pos < f.capn) {
            f.jn[rown + pos] = j;
            f.sn[rown + pos] = (uint8_t)code;
            Hn[rown + pos] = tap * P->k_e / m_cbrt(sh3);
          }
        } else {
          const int pos = cntf + __popc(mf & below);
          if (pos < f.cap) {
            f.j[rowf + pos] = j;
            f.s[rowf + pos] = (uint8_t)code;
            Hf[rowf + pos] = tap * P->k_e * f_pow(sh3, R(-1) / R(3));
          }
        }
      }
      cntn += __popc(mn);
      cntf += __popc(mf);
    }
  }
  if (lane == 0) {
    f.cntn[i] = cntn < f.capn ? cntn : f.capn;
    f.cnt[i] = cntf < f.cap ? cntf : f.cap;
    if (cntn > f.capn) atomicOr(s.err, ERR_CAP_NEAR);
    if (cntf > f.cap) atomicOr(s.err, ERR_CAP_FAR);
  }
}

// BO' components and their r-derivatives: sigma carries the (1 + bo_cut) factor.
// (r/r0)^p = exp(p log1p((r - r0)/r0)); in FP32 r and r0 are float-float so the
// difference r - r0 keeps full relative precision (steep exponents p ~ 10-40 amplify
// any relative error of r/r0 by p).
template <typename R>
__device__ __forceinline__ R pow_ratio(R rh, R rl, R r0h, R r0l, R p) {
  const R u = ((rh - r0h) + (rl - r0l)) / r0h;
  return m_exp(p * m_log1p(u));
}
template <typename R>
__device__ __forceinline__ void bo_prime(const DParams<R>* P, int pt, R r, R rl, R& bs, R& bp, R& bpp, R& dbs,
                                         R& dbp, R& dbpp) {
  bs = bp = bpp = dbs = dbp = dbpp = R(0);
  if constexpr (sizeof(R) == 8) {
    // FP64: (r/r0)^p = exp(p (log r - log r0)) with one log of r for the three components
    // (log r0 from the host); the absolute error of the log difference, ~1e-16, leaves the
    // power accurate to ~p 1e-16 relative. One reciprocal of r for the three derivatives.
    const R lr = m_log(r), ir = R(1) / r;
    if (P->r0s[pt] > R(0)) {
      const R tt = m_exp(P->p_bo2[pt] * (lr - P->lr0s[pt]));
      bs = (R(1) + P->bo_cut) * m_exp(P->p_bo1[pt] * tt);
      dbs = bs * P->p_bo1[pt] * P->p_bo2[pt] * tt * ir;
    }
    if (P->r0p[pt] > R(0)) {
      const R tt = m_exp(P->p_bo4[pt] * (lr - P->lr0p[pt]));
      bp = m_exp(P->p_bo3[pt] * tt);
      dbp = bp * P->p_bo3[pt] * P->p_bo4[pt] * tt * ir;
    }
    if (P->r0pp[pt] > R(0)) {
      const R tt = m_exp(P->p_bo6[pt] * (lr - P->lr0pp[pt]));
      bpp = m_exp(P->p_bo5[pt] * tt);
      dbpp = bpp * P->p_bo5[pt] * P->p_bo6[pt] * tt * ir;
    }
    return;
  }
  R r0 = P->r0s[pt];
  if (r0 > R(0)) {
    R tt = pow_ratio<R>(r, rl, r0, P->r0s_lo[pt], P->p_bo2[pt]);
    bs = (R(1) + P->bo_cut) * m_exp(P->p_bo1[pt] * tt);
    dbs = bs * P->p_bo1[pt] * P->p_bo2[pt] * tt / r;
  }
  r0 = P->r0p[pt];
  if (r0 > R(0)) {
    R tt = pow_ratio<R>(r, rl, r0, P->r0p_lo[pt], P->p_bo4[pt]);
    bp = m_exp(P->p_bo3[pt] * tt);
    dbp = bp * P->p_bo3[pt] * P->p_bo4[pt] * tt / r;
  }
  r0 = P->r0pp[pt];
  if (r0 > R(0)) {
    R tt = pow_ratio<R>(r, rl, r0, P->r0pp_lo[pt], P->p_bo6[pt]);
    bpp = m_exp(P->p_bo5[pt] * tt);
    dbpp = bpp * P->p_bo5[pt] * P->p_bo6[pt] * tt / r;
  }
}

// exact FP64 bond membership (used directly in FP64 mode, in the ambiguous band in FP32)
__device__ __forceinline__ bool bond_member_exact(const Sys& s, const DParams<double>* Pd, int i, int j,
                                                  int code, int r, int pt) {
  double r2 = r2_exact(s, i, j, code, r);
  if (!(r2 < Pd->r_bond * Pd->r_bond)) return false;
  double rr = sqrt(r2);
  double bs, bp, bpp, a, b, c;
  bo_prime<double>(Pd, pt, rr, 0.0, bs, bp, bpp, a, b, c);
  return bs + bp + bpp >= Pd->bo_cut;
}

// Capped at 64 registers (68 / 70 uncapped, no spills either way): 32 warps per SM instead of
// 28 for this latency-bound kernel (1,039,360 atoms: 1.09 -> 1.00 ms).
template <typename R>
__global__ void __maxnreg__(64) k_bond_list(Sys s, FarList f, BondList bl, HbList hl, AtomQ aq,
                            const DParams<R>* __restrict__ P, const DParams<double>* __restrict__ Pd, int hb_built) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= s.n) return;
  const int i = warp;
  const int r = s.rep[i];
  const int ti = s.type[i];
  const bool is_h = !hb_built && P->hb[ti] == 1;       // hb_built: the candidate filter made that list
  const int brow = i * bl.cap, hrow = i * hl.cap;
  R* bdx = (R*)bl.dx; R* bdy = (R*)bl.dy; R* bdz = (R*)bl.dz; R* br = (R*)bl.r;
  const double rh2 = Pd->r_hb * Pd->r_hb;
  int nb = 0, nh = 0;
  // near part: every entry has r < r_bond (decided exactly by the far-list pass)
  const int nn = f.cntn[i];
  const int frow = i * f.capn;
  for (int base = 0; base < nn; base += 32) {
    int k = base + lane;
    bool isb = false, ish = false;
    int j = 0, code = 0;
    R dx = 0, dy = 0, dz = 0, rr = 0;
    if (k < nn) {
      j = f.jn[frow + k];
      code = f.sn[frow + k];
      const int pt = ti * MAXT + s.type[j];
      // membership: BO'(r) >= bo_cut  <=>  r <= bcut (exact FP64 evaluation within 1e-7 A of
      // bcut, where the float-float or double distance cannot decide)
      constexpr double BAND = 1e-7;
      if (sizeof(R) == 8) {
        PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
        rr = m_sqrt(dx * dx + dy * dy + dz * dz);
        const double dr = (double)rr - Pd->bcut[pt];
        isb = (Pd->bcut_ok[pt] && dr < -BAND) ? true
              : (Pd->bcut_ok[pt] && dr > BAND) ? false
              : bond_member_exact(s, Pd, i, j, code, r, pt);
      } else {
        int sx, sy, sz;
        shift_decode(code, sx, sy, sz);
        const float* Lh = s.boxh + 3 * r;
        const float* Ll = s.boxl + 3 * r;
        float dh[3], dl[3], rh, rl;
        const float4 hj = s.ph[j], hi = s.ph[i], lj = s.pl[j], li = s.pl[i];
        pv_comp_ff(hj.x, hi.x, lj.x, li.x, sx, Lh[0], Ll[0], dh[0], dl[0]);
        pv_comp_ff(hj.y, hi.y, lj.y, li.y, sy, Lh[1], Ll[1], dh[1], dl[1]);
        pv_comp_ff(hj.z, hi.z, lj.z, li.z, sz, Lh[2], Ll[2], dh[2], dl[2]);
        norm_ff(dh, dl, rh, rl);
        dx = (R)dh[0]; dy = (R)dh[1]; dz = (R)dh[2];
        rr = (R)rh;
        const float dr = (rh - P->bcut_h[pt]) + (rl - P->bcut_l[pt]);   // exact leading difference
        isb = (P->bcut_ok[pt] && dr < -(float)BAND) ? true
              : (P->bcut_ok[pt] && dr > (float)BAND) ? false
              : bond_member_exact(s, Pd, i, j, code, r, pt);
      }
      ish = is_h && P->hb[s.type[j]] == 2;               // r < r_bond <= r_hb
    }
    const unsigned mb = __ballot_sync(0xffffffffu, isb);
    const int pos = nb + __popc(mb & ((1u << lane) - 1u));
    if (isb && pos < bl.cap) {
      const int e = brow + pos;
      bl.j[e] = j;
      bl.s[e] = (uint8_t)code;
      bdx[e] = dx; bdy[e] = dy; bdz[e] = dz; br[e] = rr;
      if ((i < j) || (i == j && code > 13)) bl.canon[atomicAdd(bl.ncanon, 1)] = e;
    }
    nb += __popc(mb);
    const unsigned mh = __ballot_sync(0xffffffffu, ish);
    const int hp = nh + __popc(mh & ((1u << lane) - 1u));
    if (ish && hp < hl.cap) {
      hl.j[hrow + hp] = j;
      hl.s[hrow + hp] = (uint8_t)code;
    }
    nh += __popc(mh);
  }
  // far part: H-bond partners with r_bond <= r < r_hb (H atoms only)
  if (is_h) {
    const int nfa = f.cnt[i];
    const int frw = i * f.cap;
    for (int base = 0; base < nfa; base += 32) {
      int k = base + lane;
      bool ish = false;
      int j = 0, code = 0;
      if (k < nfa) {
        j = f.j[frw + k];
        code = f.s[frw + k];
        if (P->hb[s.type[j]] == 2) {
          if (sizeof(R) == 8) {
            ish = r2_exact(s, i, j, code, r) < rh2;
          } else {
            R dx, dy, dz;
            PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
            const float r2f = (float)(dx * dx + dy * dy + dz * dz);
            const float m = (float)rh2 * 1e-4f;
            ish = r2f < (float)rh2 - m ? true : (r2f > (float)rh2 + m ? false : r2_exact(s, i, j, code, r) < rh2);
          }
        }
      }
      const unsigned mh = __ballot_sync(0xffffffffu, ish);
      const int hp = nh + __popc(mh & ((1u << lane) - 1u));
      if (ish && hp < hl.cap) {
        hl.j[hrow + hp] = j;
        hl.s[hrow + hp] = (uint8_t)code;
      }
      nh += __popc(mh);
    }
  }
  if (lane == 0) {
    bl.cnt[i] = nb < bl.cap ? nb : bl.cap;
    if (nb > bl.cap) atomicOr(s.err, ERR_CAP_BOND);
    if (!hb_built) {
      hl.cnt[i] = nh < hl.cap ? nh : hl.cap;
      if (nh > hl.cap) atomicOr(s.err, ERR_CAP_HB);
    }
  }
}

__global__ void k_bond_mirror(Sys s, BondList bl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  int nb = bl.cnt[i];
  for (int k = 0; k < nb; ++k) {
    int e = i * bl.cap + k;
    int j = bl.j[e];
    int want = 26 - (int)bl.s[e];
    int found = -1;
    int nj = bl.cnt[j];
    for (int m = 0; m < nj; ++m) {
      int e2 = j * bl.cap + m;
      if (bl.j[e2] == i && (int)bl.s[e2] == want) {
        found = e2;
        break;
      }
    }
    if (found < 0) {
      atomicOr(s.err, ERR_CAP_BOND);
      found = e;
    }
    bl.mirror[e] = found;
  }
}

// float hi/lo copies of the positions (every step)
__global__ void k_pos_f32(Sys s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  write_pos_f32(s, i);
}

// displacement since the last build, |(x + img L) - xb|, against skin/2
__global__ void k_skin_check(Sys s, CandList cl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double* L = s.box + 3 * s.rep[i];
  const double p[3] = {s.x[i], s.y[i], s.z[i]};
  double d2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double dd = (p[d] + s.img[3 * i + d] * L[d]) - s.xb[3 * i + d];
    d2 += dd * dd;
  }
  if (!(d2 <= cl.half_skin2)) atomicOr(s.rebuild, 1);
}

// candidate rows: every (j, image) within r_nb + skin (FP32 with a margin: a superset),
// built from the cell stencil; resets the atom's reference position and crossings.
// c.slices blocks per home cell, each taking a contiguous share of its atoms (several when
// the system has few cells, so that the grid fills the GPU): each of the 27 stencil cells is
// staged in shared memory once per block (FP32 positions and atom ids, CB_STAGE atoms per
// pass) and scanned by the block's home atoms, warp per home atom, 32 candidates per ballot. A row lists its candidates in the same order as a
// scan of the stencil atom by atom would (stencil cells in order, each cell's atoms in cell
// order), so the rows do not depend on this blocking; the staging replaces a gather of
// three coordinates per candidate and home atom by one per candidate and home cell.
constexpr int CB_THREADS = 256;
constexpr int CB_STAGE = 512;                 // stencil-cell atoms per staging pass
constexpr int CB_HOME = 256;                  // home atoms per pass (their row counts in shared memory)
__global__ void __launch_bounds__(CB_THREADS) k_cand_build(Sys s, Cells c, CandList cl) {
  if (*s.rebuild == 0) return;
  const int cell = blockIdx.x / c.slices, slice = blockIdx.x % c.slices;
  const int ca = c.start[cell], cb = c.start[cell + 1];
  const int a = ca + (int)((long long)(cb - ca) * slice / c.slices);
  const int b = ca + (int)((long long)(cb - ca) * (slice + 1) / c.slices);
  if (a >= b) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = CB_THREADS / 32;
  __shared__ float sx[CB_STAGE], sy[CB_STAGE], sz[CB_STAGE];
  __shared__ int sj[CB_STAGE];
  __shared__ int scnt[CB_HOME];
  const int r = s.rep[c.atoms[a]];
  const int* nc = c.nc + 3 * r;
  const float* Lh = s.boxh + 3 * r;
  const int lc = cell - c.cell_off[r];
  const int ci[3] = {lc % nc[0], (lc / nc[0]) % nc[1], lc / (nc[0] * nc[1])};
  for (int h0 = a; h0 < b; h0 += CB_HOME) {
    const int h1 = min(b, h0 + CB_HOME);
    for (int t = threadIdx.x; t < h1 - h0; t += CB_THREADS) scnt[t] = 0;
    for (int o = 0; o < 27; ++o) {
      const int oc[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      int t3[3], sh[3];
      for (int d = 0; d < 3; ++d) {
        const int v = ci[d] + oc[d];
        sh[d] = v < 0 ? -1 : (v >= nc[d] ? 1 : 0);
        t3[d] = v - sh[d] * nc[d];
      }
      const int code = (sh[0] + 1) * 9 + (sh[1] + 1) * 3 + (sh[2] + 1);
      const int cid = c.cell_off[r] + (t3[2] * nc[1] + t3[1]) * nc[0] + t3[0];
      const int na = c.start[cid], nb = c.start[cid + 1];
      const float ox = sh[0] * Lh[0], oy = sh[1] * Lh[1], oz = sh[2] * Lh[2];
      for (int p0 = na; p0 < nb; p0 += CB_STAGE) {
        const int np = min(CB_STAGE, nb - p0);
        __syncthreads();                          // the previous pass's readers are done
        for (int t = threadIdx.x; t < np; t += CB_THREADS) {
          const int j = c.atoms[p0 + t];
          sj[t] = j;
          sx[t] = s.xh[j];
          sy[t] = s.yh[j];
          sz[t] = s.zh[j];
        }
        __syncthreads();
        for (int h = h0 + warp; h < h1; h += nw) {
          const int i = c.atoms[h];
          const float xi = s.xh[i], yi = s.yh[i], zi = s.zh[i];
          const int row = i * cl.cap;
          int count = scnt[h - h0];                // this warp alone owns home atom h
          for (int base = 0; base < np; base += 32) {
            const int k = base + lane;
            bool ok = false;
            int j = -1;
            if (k < np) {
              j = sj[k];
              const float dx = (sx[k] - xi) + ox, dy = (sy[k] - yi) + oy, dz = (sz[k] - zi) + oz;
              ok = !(j == i && code == 13) && dx * dx + dy * dy + dz * dz < cl.rc2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            const int pos = count + __popc(m & ((1u << lane) - 1u));
            if (ok && pos < cl.cap) {
              cl.j[row + pos] = j;
              cl.s[row + pos] = (uint8_t)code;
            }
            count += __popc(m);
          }
          __syncwarp();
          if (lane == 0) scnt[h - h0] = count;
          __syncwarp();
        }
      }
    }
    __syncthreads();
    for (int h = h0 + warp; h < h1; h += nw) {
      const int i = c.atoms[h];
      const int count = scnt[h - h0];
      if (lane == 0) {
        cl.cnt[i] = count < cl.cap ? count : cl.cap;
        if (count > cl.cap) atomicOr(s.err, ERR_CAP_CAND);
      }
      if (lane < 3) {
        s.xb[3 * i + lane] = lane == 0 ? s.x[i] : (lane == 1 ? s.y[i] : s.z[i]);
        s.img[3 * i + lane] = 0;
        if (lane == 0 && s.pl) ((float*)(s.pl + i))[3] = pack_type_img(s.type[i], 0, 0, 0);
      }
    }
    __syncthreads();                              // scnt is reused by the next home pass
  }
}

// every step: exact membership (same rule as the stencil far list) over the candidates;
// image shift corrected by the box crossings since the build
template <typename R>
__global__ void k_cand_filter(Sys s, CandList cl, FarList f, HbList hl, const DParams<R>* __restrict__ P, float margin,
                              float margin_near, float margin_hb, double R2, double Rb2, double Rh2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= s.n) return;
  const int i = warp;
  const int r = s.rep[i];
  const float* Lh = s.boxh + 3 * r;
  const float R2f = (float)R2, Rb2f = (float)Rb2, Rh2f = (float)Rh2;
  const float xi = s.xh[i], yi = s.yh[i], zi = s.zh[i];
  int ii0, ii1, ii2;
  rec_img(s.pl[i].w, ii0, ii1, ii2);
  const int ti = s.type[i];
  const bool is_h = P->hb[ti] == 1;                     // H atoms also collect their H-bond partners
  const int nc = cl.cnt[i], crow = i * cl.cap;
  const int hrow = i * hl.cap;
  int cntn = 0, cntf = 0, cnth = 0;
  const int rown = i * f.capn, rowf = i * f.cap;
  R* Hn = (R*)f.Hn;
  R* Hf = (R*)f.H;
  for (int base = 0; base < nc; base += 32) {
    const int k = base + lane;
    bool ok = false, near = false, ish = false;
    int j = -1, code = 13;
    if (k < nc) {
      j = cl.j[crow + k];
      int sx, sy, sz, jx, jy, jz;
      shift_decode(cl.s[crow + k], sx, sy, sz);
      const float4 hj = s.ph[j];
      const float wj = s.pl[j].w;
      rec_img(wj, jx, jy, jz);                          // crossing counters ride in the record
      sx += jx - ii0;
      sy += jy - ii1;
      sz += jz - ii2;
      if (sx >= -1 && sx <= 1 && sy >= -1 && sy <= 1 && sz >= -1 && sz <= 1) {
        code = (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1);
        const float dx = (hj.x - xi) + sx * Lh[0], dy = (hj.y - yi) + sy * Lh[1];
        const float dz = (hj.z - zi) + sz * Lh[2];
        const float r2f = dx * dx + dy * dy + dz * dz;
        ok = !(j == i && code == 13) && in_range(s, i, j, code, r, r2f, R2f, margin, R2);
        if (ok) near = in_range(s, i, j, code, r, r2f, Rb2f, margin_near, Rb2);
        // H-bond partner: an acceptor with r < r_hb (every near pair of one is, r_bond <= r_hb)
        if (ok && is_h && P->hb[rec_type(wj)] == 2)
          ish = near || in_range(s, i, j, code, r, r2f, Rh2f, margin_hb, Rh2);
      }
    }
    const unsigned mn = __ballot_sync(0xffffffffu, ok && near);
    const unsigned mf = __ballot_sync(0xffffffffu, ok && !near);
    const unsigned mh = __ballot_sync(0xffffffffu, ish);
    const unsigned below = (1u << lane) - 1u;
    if (ish) {
      const int hp = cnth + __popc(mh & below);
      if (hp < hl.cap) {
        hl.j[hrow + hp] = j;
        hl.s[hrow + hp] = (uint8_t)code;
      }
    }
    cnth += __popc(mh);
    if (ok) {
      R dx, dy, dz;
      int tj;
      if constexpr (sizeof(R) == 4) {
        float4 hj, lj;
        PairVec<float>::getv(s, i, j, code, r, dx, dy, dz, hj, lj);
        tj = rec_type(lj.w);
      } else {
        PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
        tj = s.type[j];
      }
      const R rr = m_sqrt(dx * dx + dy * dy + dz * dz);
      R tap, dtap;
      taper<R>(rr, P->r_nb, tap, dtap);
      const R sh3 = rr * rr * rr + P->gamma_m3[ti * MAXT + tj];
      if (near) {
        const int pos = cntn + __popc(mn & below);
        if (pos < f.capn) {
          f.jn[rown + pos] = j;
          f.sn[rown + pos] = (uint8_t)code;
          Hn[rown + pos] = tap * P->k_e / m_cbrt(sh3);
        }
      } else {
        const int pos = cntf + __popc(mf & below);
        if (pos < f.cap) {
          f.j[rowf + pos] = j;
          f.s[rowf + pos] = (uint8_t)code;
          Hf[rowf + pos] = tap * P->k_e * f_pow(sh3, R(-1) / R(3));
        }
      }
    }
    cntn += __popc(mn);
    cntf += __popc(mf);
  }
  if (lane == 0) {
    f.cntn[i] = cntn < f.capn ? cntn : f.capn;
    f.cnt[i] = cntf < f.cap ? cntf : f.cap;
    hl.cnt[i] = cnth < hl.cap ? cnth : hl.cap;
    if (cntn > f.capn) atomicOr(s.err, ERR_CAP_NEAR);
    if (cntf > f.cap) atomicOr(s.err, ERR_CAP_FAR);
    if (cnth > hl.cap) atomicOr(s.err, ERR_CAP_HB);
  }
}

__global__ void k_rebuild_done(Sys s) {
  if (threadIdx.x == 0) *s.rebuild = 0;
}

// FP64 BO' of each unordered bond (thread per bond), written to both directed entries
__global__ void k_bo_prime64(Sys s, BondList bl, const DParams<double>* __restrict__ P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *bl.ncanon) return;
  const int e = bl.canon[t];
  const int i = e / bl.cap;
  const int j = bl.j[e];
  const int code = bl.s[e];
  double dx, dy, dz;
  PairVec<double>::get(s, i, j, code, s.rep[i], dx, dy, dz);
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double bs, bp, bpp, dbs, dbp, dbpp;
  bo_prime<double>(P, s.type[i] * MAXT + s.type[j], r, 0.0, bs, bp, bpp, dbs, dbp, dbpp);
  const int m = bl.mirror[e];
  const double tot = bs + bp + bpp - P->bo_cut;
  bl.bop[e] = tot; bl.bopi[e] = bp; bl.bopp[e] = bpp;
  bl.dbop[e] = dbs + dbp + dbpp; bl.dbopi[e] = dbp; bl.dbopp[e] = dbpp;
  bl.bop[m] = tot; bl.bopi[m] = bp; bl.bopp[m] = bpp;
  bl.dbop[m] = dbs + dbp + dbpp; bl.dbopi[m] = dbp; bl.dbopp[m] = dbpp;
}

// Delta'_i = sum BO'_ij - Val_i and Delta'boc_i (FP64, in row order)
__global__ void k_delta_prime(Sys s, BondList bl, AtomQ aq, const DParams<double>* __restrict__ P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  double sum = 0.0;
  for (int k = 0; k < bl.cnt[i]; ++k) sum += bl.bop[i * bl.cap + k];
  aq.dp[i] = sum - P->val[s.type[i]];
  aq.dpboc[i] = sum - P->valboc[s.type[i]];
}

inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }

// 1/cbrt(x) for x > 0: the MUFU estimate 2^(-log2(x)/3) (relative error ~1e-6) and one
// Newton step on y^-3 = x, y <- y + y (1 - x y^3) / 3, which squares the relative error
__device__ __forceinline__ float rcbrt_f(float x) {
  const float y = __powf(x, -1.0f / 3.0f);
  const float y3 = y * y * y;
  const float e = __fmaf_rn(-x, y3, 1.0f);
  return __fmaf_rn(y * (1.0f / 3.0f), e, y);
}

// Mixed path form of k_cand_filter: atom i's records, box and image counters live in
// registers; the shift code is decoded once; atom j's two 16-byte records are read once and
// give the FP32 image vector used both for the range decisions (its error is far inside the
// margins) and for H; H = Tap(r) k_e (r^3 + gamma^-3)^(-1/3) with one
// branch-free rcbrt_f for near and far entries; the near/far destination is a per-lane
// select, so the stores do not diverge. Capped at 56 registers (54 used, no spills; 63
// uncapped): 36 warps per SM instead of 32 for this latency-bound kernel (petn32k filter
// 0.176 -> 0.172 ms).
__global__ void __maxnreg__(56) k_cand_filter_f(Sys s, CandList cl, FarList f, HbList hl, const DParams<float>* __restrict__ P,
                                float margin, float margin_near, float margin_hb, double R2, double Rb2, double Rh2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= s.n) return;
  const int i = warp;
  const int r = s.rep[i];
  const float Lh0 = s.boxh[3 * r], Lh1 = s.boxh[3 * r + 1], Lh2 = s.boxh[3 * r + 2];
  const float Ll0 = s.boxl[3 * r], Ll1 = s.boxl[3 * r + 1], Ll2 = s.boxl[3 * r + 2];
  const float R2f = (float)R2, Rb2f = (float)Rb2, Rh2f = (float)Rh2;
  const float4 hi = s.ph[i], li = s.pl[i];
  int ii0, ii1, ii2;
  rec_img(li.w, ii0, ii1, ii2);
  const int ti = s.type[i];
  unsigned acc = 0;                                     // acceptor types, when i is an H-bond H
  if (P->hb[ti] == 1)
    for (int t = 0; t < MAXT; ++t) acc |= (P->hb[t] == 2 ? 1u : 0u) << t;
  const float irnb = 1.0f / P->r_nb, ke = P->k_e;
  const float* gam = P->gamma_m3 + ti * MAXT;
  const int nc = cl.cnt[i], crow = i * cl.cap;
  const int hrow = i * hl.cap;
  int cntn = 0, cntf = 0, cnth = 0;
  const int rown = i * f.capn, rowf = i * f.cap;
  float* Hn = (float*)f.Hn;
  float* Hf = (float*)f.H;
  for (int base = 0; base < nc; base += 32) {
    const int k = base + lane;
    bool ok = false, near = false, ish = false;
    int j = -1, code = 13, tj = 0;
    float r2f = 0.f;
    if (k < nc) {
      j = cl.j[crow + k];
      const int c0 = cl.s[crow + k];
      const float4 hj = s.ph[j], lj = s.pl[j];
      int jx, jy, jz;
      rec_img(lj.w, jx, jy, jz);                        // crossing counters ride in the record
      const int sx = c0 / 9 - 1 + jx - ii0, sy = (c0 / 3) % 3 - 1 + jy - ii1, sz = c0 % 3 - 1 + jz - ii2;
      if (sx >= -1 && sx <= 1 && sy >= -1 && sy <= 1 && sz >= -1 && sz <= 1) {
        code = (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1);
        tj = rec_type(lj.w);
        // plain FP32 image vector (hi difference + lo difference, image shift by exact
        // products): |error of r^2| <= u (3.5 r L_max + 8 r^2), inside the decision margins
        // 32 u (L_max R + R^2) by a factor of ~8; pairs inside a margin are decided in FP64
        const float fx = (float)sx, fy = (float)sy, fz = (float)sz;
        const float dx = fmaf(fx, Lh0, hj.x - hi.x) + fmaf(fx, Ll0, lj.x - li.x);
        const float dy = fmaf(fy, Lh1, hj.y - hi.y) + fmaf(fy, Ll1, lj.y - li.y);
        const float dz = fmaf(fz, Lh2, hj.z - hi.z) + fmaf(fz, Ll2, lj.z - li.z);
        r2f = dx * dx + dy * dy + dz * dz;
        ok = !(j == i && code == 13) && in_range(s, i, j, code, r, r2f, R2f, margin, R2);
        if (ok) near = in_range(s, i, j, code, r, r2f, Rb2f, margin_near, Rb2);
        // H-bond partner: an acceptor with r < r_hb (every near pair of one is, r_bond <= r_hb)
        if (ok && ((acc >> tj) & 1u)) ish = near || in_range(s, i, j, code, r, r2f, Rh2f, margin_hb, Rh2);
      }
    }
    const unsigned mn = __ballot_sync(0xffffffffu, ok && near);
    const unsigned mf = __ballot_sync(0xffffffffu, ok && !near);
    const unsigned mh = __ballot_sync(0xffffffffu, ish);
    const unsigned below = (1u << lane) - 1u;
    if (ish) {
      const int hp = cnth + __popc(mh & below);
      if (hp < hl.cap) {
        hl.j[hrow + hp] = j;
        hl.s[hrow + hp] = (uint8_t)code;
      }
    }
    cnth += __popc(mh);
    if (ok) {
      // r from the MUFU reciprocal square root (relative error ~1e-7, far inside what the
      // solve tolerance allows for H) and x = r / r_nb by the reciprocal cutoff
      const float rr = r2f * rsqrtf(r2f);
      const float x = rr * irnb, x2 = x * x;
      const float tap = ((((20.0f * x - 70.0f) * x + 84.0f) * x - 35.0f) * x2 * x2) + 1.0f;
      const float h = tap * ke * rcbrt_f(rr * r2f + gam[tj]);
      const int pos = near ? cntn + __popc(mn & below) : cntf + __popc(mf & below);
      if (pos < (near ? f.capn : f.cap)) {
        const int e = (near ? rown : rowf) + pos;
        (near ? f.jn : f.j)[e] = j;
        (near ? f.sn : f.s)[e] = (uint8_t)code;
        (near ? Hn : Hf)[e] = h;
      }
    }
    cntn += __popc(mn);
    cntf += __popc(mf);
  }
  if (lane == 0) {
    f.cntn[i] = cntn < f.capn ? cntn : f.capn;
    f.cnt[i] = cntf < f.cap ? cntf : f.cap;
    hl.cnt[i] = cnth < hl.cap ? cnth : hl.cap;
    if (cntn > f.capn) atomicOr(s.err, ERR_CAP_NEAR);
    if (cntf > f.cap) atomicOr(s.err, ERR_CAP_FAR);
    if (cnth > hl.cap) atomicOr(s.err, ERR_CAP_HB);
  }
}

}  // namespace

namespace rx {

void cells_build(const Launch& L, Sys s, Cells c) {
  cudaMemsetAsync(c.count, 0, sizeof(int) * c.ncell_total, L.st);
  k_cell_assign<false><<<grid_for(s.n, 256), 256, 0, L.st>>>(s, c);
  k_cell_scan<false><<<1, 1024, 0, L.st>>>(c, nullptr);
  k_cell_scatter<false><<<grid_for(s.n, 256), 256, 0, L.st>>>(s, c, c.tmp);
  k_cell_sort<false><<<c.ncell_total, 128, 0, L.st>>>(c, c.tmp, nullptr);
  *L.count += 4;
}

void positions_f32(const Launch& L, Sys s) {
  k_pos_f32<<<grid_for(s.n, 256), 256, 0, L.st>>>(s);
  *L.count += 1;
}

void skin_check(const Launch& L, Sys s, CandList cl) {
  k_skin_check<<<grid_for(s.n, 256), 256, 0, L.st>>>(s, cl);
  *L.count += 1;
}

void cand_build(const Launch& L, Sys s, Cells c, CandList cl) {
  cudaMemsetAsync(c.count, 0, sizeof(int) * c.ncell_total, L.st);
  k_cell_assign<true><<<grid_for(s.n, 256), 256, 0, L.st>>>(s, c);
  k_cell_scan<true><<<1, 1024, 0, L.st>>>(c, s.rebuild);
  k_cell_scatter<true><<<grid_for(s.n, 256), 256, 0, L.st>>>(s, c, c.tmp);
  k_cell_sort<true><<<c.ncell_total, 128, 0, L.st>>>(c, c.tmp, s.rebuild);
  k_cand_build<<<c.ncell_total * c.slices, CB_THREADS, 0, L.st>>>(s, c, cl);
  *L.count += 5;
}

template <typename R>
void cand_filter(const Launch& L, Sys s, CandList cl, FarList f, HbList h, const DParams<R>* P, float margin,
                 float margin_near, float margin_hb) {
  const int bs = L.t().cf_block;
  if constexpr (sizeof(R) == 4)
    k_cand_filter_f<<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, cl, f, h, P, margin, margin_near,
                                                                        margin_hb, f.r2_nb, f.r2_bond, f.r2_hb);
  else
    k_cand_filter<R><<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, cl, f, h, P, margin, margin_near,
                                                                           margin_hb, f.r2_nb, f.r2_bond, f.r2_hb);
  k_rebuild_done<<<1, 32, 0, L.st>>>(s);
  *L.count += 2;
}
template void cand_filter<double>(const Launch&, Sys, CandList, FarList, HbList, const DParams<double>*, float, float,
                                  float);
template void cand_filter<float>(const Launch&, Sys, CandList, FarList, HbList, const DParams<float>*, float, float,
                                 float);

template <typename R>
void far_list(const Launch& L, Sys s, Cells c, FarList f, const DParams<R>* P, float margin) {
  k_far_list<R><<<grid_for((long long)s.n * 32, 256), 256, 0, L.st>>>(s, c, f, P, margin);
  *L.count += 1;
}

template <typename R>
void far_list_split(const Launch& L, Sys s, Cells c, FarList f, const DParams<R>* P, float margin,
                    float margin_near) {
  k_far_list_split<R><<<grid_for((long long)s.n * 32, 256), 256, 0, L.st>>>(s, c, f, P, margin, margin_near,
                                                                           f.r2_nb, f.r2_bond);
  *L.count += 1;
}

template <typename R>
void bond_list(const Launch& L, Sys s, FarList f, BondList b, HbList h, AtomQ a, const DParams<R>* P,
               const DParams<double>* Pd, bool hb_built) {
  const int bs = L.t().bl_block;
  k_bond_list<R><<<grid_for((long long)s.n * 32, bs), bs, 0, L.st>>>(s, f, b, h, a, P, Pd, hb_built ? 1 : 0);
  *L.count += 1;
}

namespace {
__global__ void k_q_to_f32(Sys s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s.n) write_q_f32(s, i, s.q[i]);
}
}  // namespace
void charges_to_f32(const Launch& L, Sys s) {
  k_q_to_f32<<<grid_for(s.n, 256), 256, 0, L.st>>>(s);
  *L.count += 1;
}

void bond_mirror(const Launch& L, Sys s, BondList b) {
  k_bond_mirror<<<grid_for(s.n, 128), 128, 0, L.st>>>(s, b);
  *L.count += 1;
}

void bo_prime64(const Launch& L, Sys s, BondList b, AtomQ a, const DParams<double>* Pd, int n_canon_max) {
  k_bo_prime64<<<grid_for(n_canon_max, 128), 128, 0, L.st>>>(s, b, Pd);
  k_delta_prime<<<grid_for(s.n, 128), 128, 0, L.st>>>(s, b, a, Pd);
  *L.count += 2;
}

template void far_list<double>(const Launch&, Sys, Cells, FarList, const DParams<double>*, float);
template void far_list<float>(const Launch&, Sys, Cells, FarList, const DParams<float>*, float);
template void far_list_split<double>(const Launch&, Sys, Cells, FarList, const DParams<double>*, float, float);
template void far_list_split<float>(const Launch&, Sys, Cells, FarList, const DParams<float>*, float, float);
template void bond_list<double>(const Launch&, Sys, FarList, BondList, HbList, AtomQ, const DParams<double>*,
                                const DParams<double>*, bool);
template void bond_list<float>(const Launch&, Sys, FarList, BondList, HbList, AtomQ, const DParams<float>*,
                               const DParams<double>*, bool);
}  // namespace rx

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

template <typename R>
__global__ void k_nonbonded(Sys s, FarList f, Accum acc, const DParams<R>* __restrict__ P, unsigned mask) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= s.n) return;
  const int ti = s.type[i];
  const int r = s.rep[i];
  const int nf = f.cnt[i];
  const int row = i * f.cap;
  const R qi = (R)s.q[i];
  const R wv = ((mask >> T_VDW) & 1u) ? R(1) : R(0);
  const R wc = ((mask >> T_COUL) & 1u) ? R(1) : R(0);
  const R pv = P->p_vdW1, ipv = R(1) / P->p_vdW1;
  double ev = 0, ec = 0, fx = 0, fy = 0, fz = 0, w[6] = {0, 0, 0, 0, 0, 0};
  for (int k = lane; k < nf; k += 32) {
    const int j = f.j[row + k];
    const int code = f.s[row + k];
    R dx, dy, dz;
    PairVec<R>::get(s, i, j, code, r, dx, dy, dz);
    const R r2 = dx * dx + dy * dy + dz * dz;
    const R rr = m_sqrt(r2);
    R tap, dtap;
    taper<R>(rr, P->r_nb, tap, dtap);
    const int pt = ti * MAXT + s.type[j];
    // van der Waals
    const R rp = m_pow(rr, pv);
    const R base = rp + P->vdw_gw_pow[pt];
    const R f13 = m_pow(base, ipv);
    const R df13 = f13 * rp / (rr * base);
    const R al = P->vdw_alpha[pt], rv = P->vdw_rv[pt], D = P->vdw_D[pt];
    const R xr = R(1) - f13 / rv;
    const R E1 = m_exp(al * xr), E2 = m_exp(R(0.5) * al * xr);
    const R evp = D * (E1 - R(2) * E2);
    const R devp = -(D * al / rv) * (E1 - E2);
    // Coulomb
    const R sh3 = r2 * rr + P->gamma_m3[pt];
    const R sh = m_cbrt(sh3);
    const R kq = P->k_e * qi * (R)s.q[j];
    const R ecp = kq / sh;
    const R decp = -kq * r2 / (sh3 * sh);
    ev += (double)(tap * evp);
    ec += (double)(tap * ecp);
    const R de = wv * (dtap * evp + tap * devp * df13) + wc * (dtap * ecp + tap * decp);
    const R c = de / rr;                                // F_i += (dE/dr) d/r
    fx += (double)(c * dx);
    fy += (double)(c * dy);
    fz += (double)(c * dz);
    // half of W_ab = -dE/dr d_a d_b / r for this direction
    const double hc = -0.5 * (double)c;
    w[0] += hc * (double)(dx * dx); w[1] += hc * (double)(dy * dy); w[2] += hc * (double)(dz * dz);
    w[3] += hc * (double)(dx * dy); w[4] += hc * (double)(dx * dz); w[5] += hc * (double)(dy * dz);
  }
  ev = warp_sum(ev); ec = warp_sum(ec);
  fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
  for (int q = 0; q < 6; ++q) w[q] = warp_sum(w[q]);
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

}  // namespace

namespace rx {
template <typename R>
void nonbonded(const Launch& L, Sys s, FarList f, Accum acc, const DParams<R>* P, unsigned mask) {
  k_nonbonded<R><<<grid_for((long long)s.n * 32, 256), 256, 0, L.st>>>(s, f, acc, P, mask);
  *L.count += 1;
}
template void nonbonded<double>(const Launch&, Sys, FarList, Accum, const DParams<double>*, unsigned);
template void nonbonded<float>(const Launch&, Sys, FarList, Accum, const DParams<float>*, unsigned);
}  // namespace rx

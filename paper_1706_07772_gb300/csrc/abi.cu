// C ABI of the library (include/reaxff.h): context, device memory plan, stage
// orchestration of one timestep, list-overflow regrow, error reporting.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <array>
#include <vector>

#include "reax_internal.cuh"

constexpr int ETOT_CHUNK = 256;   // steps per batch of device-side total energies

std::string cuda_err_str(cudaError_t e) { return std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e); }

namespace {
struct DevBuf {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <typename T> T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      err = e;
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
  void* alloc_bytes(size_t bytes) { return alloc<char>(bytes); }
  void free_all() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};
}  // namespace

struct reaxff_ctx {
  std::string err;
  int n = 0, nrep = 0;
  reaxff_params hp;
  reaxff_options ho;
  bool fp64 = true;
  unsigned mask = 0x1fff;
  int nsm = 0;
  cudaStream_t st = nullptr;
  cudaStream_t st2 = nullptr;  // second stream (highest priority): bonded terms beside the
                               // nonbonded kernel, or the QEq solve beside the charge-free terms
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t st3 = nullptr;  // third stream: the torsion kernel beside the angle and H-bond
                               // kernels inside the charge-free path (mixed path)
  cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
  int64_t launches = 0;
  bool have_pos = false, forces_valid = false, lists_valid = false;
  float far_margin = 0.f;
  std::vector<int64_t> h_rep_off;
  std::vector<double> h_box;
  std::vector<int> h_types;      // per atom, in storage order
  // storage order (options.spatial_sort): perm[k] = the caller's index of the atom stored at
  // k; empty = the caller's order
  bool sort_on = false;
  std::vector<int> perm, h_types_ext;
  int* type_d = nullptr;
  // device memory: fixed part and list part (re-allocated on regrow)
  DevBuf fixed, lists;
  DParams<double>* Pd = nullptr;
  DParams<float>* Pf = nullptr;
  Sys sys{};
  Cells cells{};
  FarList far{};
  BondList bond{};
  HbList hb{};
  AtomQ aq{};
  Accum acc{};
  rx::QeqState Q{};
  rx::RedPlan red{};
  double *F_out = nullptr, *E_rep = nullptr, *vir_rep = nullptr, *ke_rep = nullptr, *Etot_dev = nullptr;
  double* h_etot = nullptr;    // pinned copy of Etot_dev for reaxff_step
  int Etot_cap = 0;
  double *chi_t = nullptr, *eta_t = nullptr, *mass_t = nullptr;
  int* h_err_pinned = nullptr;
  // device-side state I/O (contexts in the caller's order): interleaved input and output
  // rows, the SoA staging of an upload, and a flag word (allocated on first use)
  double* d_io = nullptr;      // [13n]: x in [3n], v in [3n], SoA stage [6n]; output x, v, q [7n]
  int* d_io_flag = nullptr;
  int* h_io_flag = nullptr;    // pinned
  // host I/O: pinned staging for the state copies (6n doubles: x, y, z, vx, vy, vz as SoA,
  // allocated on first use) and the device positions as last uploaded or downloaded, valid
  // until a step moves the atoms (a round trip of unchanged positions then keeps forces,
  // lists and image counters)
  double* h_stage = nullptr;
  std::vector<double> h_pos;
  bool h_pos_valid = false;
  int cap_far = 0, cap_bond = 0, cap_hb = 0, cap_near = 0, cap_cand = 0;
  float near_margin = 0.f, hb_margin = 0.f;
  bool use_skin = true;
  double skin = 0.7;
  CandList cand{};
  // MD steps without host synchronisation: one CUDA graph per step (captured on first use,
  // dropped when the list buffers, dt or the profiling switch change), flags checked once
  // per call; a call that overflowed a list capacity is rolled back from a snapshot
  cudaGraphExec_t gexec = nullptr;
  bool capturing = false;      // inside a step capture: stage events become graph nodes
  bool graph_ok = true;        // capture works here (else the steps are launched directly)
  double g_dt = 0.0;
  int g_prof = 0;
  int64_t g_launches = 0;
  std::vector<std::pair<int, int>> g_events;
  double* etot_buf = nullptr;  // [ETOT_CHUNK * nrep] per-step total energies
  int* etot_idx = nullptr;     // device step index into etot_buf
  double* snap = nullptr;      // x, v (6n) and the QEq rings (7n)
  int* snap_i = nullptr;       // the rings' state (4)
  // learned QEq warm start (allocated on first use)
  struct Mlp {
    bool alloc = false, ready = false, fresh = false;
    DevBuf buf, data;
    float *theta = nullptr, *mean = nullptr, *inv = nullptr, *madam = nullptr, *vadam = nullptr, *grad = nullptr;
    double* loss = nullptr;
    float *D = nullptr, *y = nullptr;      // descriptors and predictions at the current positions
    int* types = nullptr;                  // [n] element of each atom
    int* off = nullptr;                    // [5] element offsets into tiles.perm
    rx::MlpTiles tiles{};
    rx::MlpInfer inf{};
    rx::MlpScratch scr{};
    int adam_step = 0;
    int cap = 0, count = 0;                // training snapshots
    float *TD = nullptr, *TQ = nullptr;
  } mlp;
  rx::Tune tune{};              // launch schedules (reaxff_autotune)
  // species analysis buffers (allocated on first use)
  DevBuf spbuf;
  rx::SpeciesBuf sp{};
  double* sp_thr = nullptr;
  DevBuf avgbuf;               // time-averaged bond orders
  rx::BoAvg avg{};
  int64_t avg_samples = 0;
  // per-stage CUDA-event timing (reaxff_profile_*)
  int prof = 0;                // 0 off; 1 stage timers (serial order); 2 overlap path spans
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pending;   // (stage, index of start event; end = +1)
  double stage_ms[32] = {0};
  int64_t stage_calls[32] = {0};
};

namespace {

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e__ = (call);                                           \
    if (e__ != cudaSuccess) {                                           \
      ctx->err = std::string(#call) + " -> " + cuda_err_str(e__);       \
      return REAXFF_E_CUDA;                                             \
    }                                                                   \
  } while (0)

int fail(reaxff_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

template <typename R> void fill_params(DParams<R>& d, const reaxff_params& p, const reaxff_options& o) {
  memset(&d, 0, sizeof(d));
  d.nt = p.ntypes;
  for (int a = 0; a < MAXT; ++a) {
    d.hb[a] = p.hb[a];
    d.mass[a] = (R)p.mass[a]; d.val[a] = (R)p.val[a]; d.vale[a] = (R)p.vale[a];
    d.valboc[a] = (R)p.valboc[a]; d.valang[a] = (R)p.valang[a]; d.p_lp2[a] = (R)p.p_lp2[a];
    d.p_ovun2[a] = (R)p.p_ovun2[a]; d.p_ovun5[a] = (R)p.p_ovun5[a]; d.p_val3[a] = (R)p.p_val3[a];
    d.p_val5[a] = (R)p.p_val5[a]; d.chi[a] = (R)p.chi[a]; d.eta[a] = (R)p.eta[a];
    for (int b = 0; b < MAXT; ++b) {
      const int k = a * MAXT + b;
#define PP(f) d.f[k] = (R)p.f[a][b]
      PP(r0s); PP(r0p); PP(r0pp); PP(p_bo1); PP(p_bo2); PP(p_bo3); PP(p_bo4); PP(p_bo5); PP(p_bo6);
      PP(p_boc3); PP(p_boc4); PP(p_boc5); PP(ovc); PP(v13); PP(De_s); PP(De_p); PP(De_pp);
      PP(p_be1); PP(p_be2); PP(p_ovun1); PP(vdw_D); PP(vdw_rv); PP(vdw_alpha);
      PP(V1); PP(V2); PP(V3); PP(p_tor1); PP(p_cot1); PP(r0hb); PP(p_hb1); PP(p_hb2); PP(p_hb3);
#undef PP
      d.vdw_gw_pow[k] = (R)std::pow(p.vdw_gw[a][b], -p.p_vdW1);
      d.r0s_lo[k] = (R)(p.r0s[a][b] - (double)(R)p.r0s[a][b]);
      d.r0p_lo[k] = (R)(p.r0p[a][b] - (double)(R)p.r0p[a][b]);
      d.r0pp_lo[k] = (R)(p.r0pp[a][b] - (double)(R)p.r0pp[a][b]);
      d.lr0s[k] = p.r0s[a][b] > 0 ? (R)std::log(p.r0s[a][b]) : R(0);
      d.lr0p[k] = p.r0p[a][b] > 0 ? (R)std::log(p.r0p[a][b]) : R(0);
      d.lr0pp[k] = p.r0pp[a][b] > 0 ? (R)std::log(p.r0pp[a][b]) : R(0);
      d.gamma_m3[k] = (R)std::pow(p.gamma[a][b], -3.0);
      {
        R* t = d.nbf + 8 * k;
        const double al = p.vdw_alpha[a][b], rv = p.vdw_rv[a][b], D = p.vdw_D[a][b];
        t[0] = (R)std::pow(p.vdw_gw[a][b], -p.p_vdW1);
        t[1] = (R)(al * 1.4426950408889634);
        t[2] = (R)(1.0 / rv);
        t[3] = (R)D;
        t[4] = (R)std::pow(p.gamma[a][b], -3.0);
        t[5] = (R)(-D * al / rv);
      }
      for (int c = 0; c < MAXT; ++c) {
        const int t3 = (a * MAXT + b) * MAXT + c;
        d.th00[t3] = (R)p.th00[a][b][c]; d.p_val1[t3] = (R)p.p_val1[a][b][c];
        d.p_val2[t3] = (R)p.p_val2[a][b][c]; d.p_val4[t3] = (R)p.p_val4[a][b][c];
        d.p_val7[t3] = (R)p.p_val7[a][b][c]; d.p_pen1[t3] = (R)p.p_pen1[a][b][c];
        d.p_coa1[t3] = (R)p.p_coa1[a][b][c];
      }
    }
  }
#define PG(f) d.f = (R)p.f
  PG(p_boc1); PG(p_boc2); PG(p_lp1); PG(p_ovun3); PG(p_ovun4); PG(p_ovun6); PG(p_ovun7); PG(p_ovun8);
  PG(p_val6); PG(p_val8); PG(p_val9); PG(p_val10); PG(p_pen2); PG(p_pen3); PG(p_pen4); PG(p_coa2);
  PG(p_coa3); PG(p_coa4); PG(p_tor2); PG(p_tor3); PG(p_tor4); PG(p_cot2); PG(p_vdW1); PG(k_e);
#undef PG
  d.r_nb = (R)o.r_nb; d.r_bond = (R)o.r_bond; d.r_hb = (R)o.r_hb; d.bo_cut = (R)o.bo_cut;
  d.thb_cut = (R)o.thb_cut; d.thb_cutsq = (R)o.thb_cutsq; d.hb_bo_min = (R)o.hb_bo_min;
  // the distance at which BO'(r) = bo_cut, per type pair (bisection in FP64 after checking
  // that BO' decreases over (0, r_bond]); the kernels decide membership by comparing r with
  // it and evaluate BO' in FP64 only within a tiny band around it
  for (int a = 0; a < MAXT; ++a)
    for (int b = 0; b < MAXT; ++b) {
      const int k = a * MAXT + b;
      auto bop = [&](double r) {
        double t = 0.0;
        if (p.r0s[a][b] > 0) t += (1.0 + o.bo_cut) * std::exp(p.p_bo1[a][b] * std::pow(r / p.r0s[a][b], p.p_bo2[a][b]));
        if (p.r0p[a][b] > 0) t += std::exp(p.p_bo3[a][b] * std::pow(r / p.r0p[a][b], p.p_bo4[a][b]));
        if (p.r0pp[a][b] > 0) t += std::exp(p.p_bo5[a][b] * std::pow(r / p.r0pp[a][b], p.p_bo6[a][b]));
        return t;
      };
      bool mono = a < p.ntypes && b < p.ntypes;
      double prev = bop(1e-3);
      for (int q = 1; q <= 2000 && mono; ++q) {
        const double v = bop(1e-3 + (o.r_bond - 1e-3) * q / 2000.0);
        if (v > prev) mono = false;
        prev = v;
      }
      double cut = 0.0;
      if (mono) {
        if (bop(o.r_bond) >= o.bo_cut) cut = o.r_bond * 2.0;          // every near pair bonds
        else if (bop(1e-3) < o.bo_cut) cut = 0.0;                      // none does
        else {
          double lo = 1e-3, hi = o.r_bond;
          for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (bop(mid) >= o.bo_cut) lo = mid; else hi = mid;
          }
          cut = 0.5 * (lo + hi);
        }
      }
      d.bcut[k] = cut;
      d.bcut_h[k] = (float)cut;
      d.bcut_l[k] = (float)(cut - (double)(float)cut);
      d.bcut_ok[k] = mono ? 1 : 0;
    }
}

int round_up(double v, int m) { return (int)((std::ceil(v) + m - 1) / m) * m; }

}  // namespace

// parameter tables in FP64 device layout (used by the allocation-free list builder)
void rx_fill_params_double(DParams<double>& d, const reaxff_params& p, const reaxff_options& o) {
  fill_params<double>(d, p, o);
}

namespace {

// allocate the three lists at the current capacities
void drop_graph(reaxff_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
}

int alloc_lists(reaxff_ctx* ctx) {
  drop_graph(ctx);
  ctx->lists.free_all();
  DevBuf& B = ctx->lists;
  const size_t n = ctx->n;
  const size_t rs = ctx->fp64 ? sizeof(double) : sizeof(float);
  FarList& f = ctx->far;
  f.cap = ctx->cap_far;
  f.cnt = B.alloc<int>(n);
  f.j = B.alloc<int>(n * f.cap);
  f.s = B.alloc<uint8_t>(n * f.cap);
  f.H = B.alloc_bytes(n * f.cap * rs);
  f.capn = ctx->cap_near;
  f.cntn = B.alloc<int>(n);
  f.jn = B.alloc<int>(n * f.capn);
  f.sn = B.alloc<uint8_t>(n * f.capn);
  f.Hn = B.alloc_bytes(n * f.capn * rs);
  f.r2_nb = ctx->ho.r_nb * ctx->ho.r_nb;
  f.r2_bond = ctx->ho.r_bond * ctx->ho.r_bond;
  f.r2_hb = ctx->ho.r_hb * ctx->ho.r_hb;
  BondList& b = ctx->bond;
  b.cap = ctx->cap_bond;
  const size_t nb = n * b.cap;
  b.cnt = B.alloc<int>(n);
  b.j = B.alloc<int>(nb);
  b.s = B.alloc<uint8_t>(nb);
  b.mirror = B.alloc<int>(nb);
  b.canon = B.alloc<int>(nb);
  b.ncanon = B.alloc<int>(1);
  void** rfields[] = {&b.dx, &b.dy, &b.dz, &b.r, &b.bo, &b.bo_pi, &b.bo_pp};
  for (void** p : rfields) *p = B.alloc_bytes(nb * rs);
  double** bofields[] = {&b.bop, &b.bopi, &b.bopp, &b.dbop, &b.dbopi, &b.dbopp};
  for (double** p : bofields) *p = B.alloc<double>(nb);
  void** dfields[] = {&b.f1, &b.fo, &b.ft, &b.df1, &b.dfo_bo, &b.dft_bo, &b.dfo_d};   // FP64 in both modes
  for (void** p : dfields) *p = B.alloc_bytes(nb * sizeof(double));
  b.dEdBOp = B.alloc<double>(nb);
  b.dEdBOpi = B.alloc<double>(nb);
  b.dEdBOpp = B.alloc<double>(nb);
  b.cdbo = B.alloc<unsigned long long>(nb);
  b.cdbopi = B.alloc<unsigned long long>(nb);
  b.cdbopp = B.alloc<unsigned long long>(nb);
  CandList& cl = ctx->cand;
  cl.cap = ctx->cap_cand;
  cl.cnt = B.alloc<int>(n);
  cl.j = B.alloc<int>(n * (size_t)cl.cap);
  cl.s = B.alloc<uint8_t>(n * (size_t)cl.cap);
  HbList& h = ctx->hb;
  h.cap = ctx->cap_hb;
  h.cnt = B.alloc<int>(n);
  h.j = B.alloc<int>(n * h.cap);
  h.s = B.alloc<uint8_t>(n * h.cap);
  if (B.err != cudaSuccess) return fail(ctx, REAXFF_E_CUDA, "list allocation: " + cuda_err_str(B.err));
  ctx->lists_valid = false;
  return REAXFF_OK;
}

rx::Launch launch_of(reaxff_ctx* ctx) { return rx::Launch{ctx->st, &ctx->launches, &ctx->tune}; }

const char* const STAGE_NAMES[] = {"cells", "far_list", "bond_list", "bo_prime64", "qeq", "bo_correct",
                                   "atom_terms", "over_under_bond", "s_gather", "angles", "torsions",
                                   "hbonds", "nonbonded", "chain_rule", "verlet", "reduce", "mlp_guess",
                                   "qeq_precond", "solve_path", "terms_path"};
constexpr int NSTAGES = 20;
constexpr int STAGE_SOLVE_PATH = 18, STAGE_TERMS_PATH = 19;

// scoped event pair around one stage (only when profiling is on)
struct Stage {
  reaxff_ctx* ctx;
  int id, idx = -1;
  Stage(reaxff_ctx* c, int s) : ctx(c), id(s) {
    if (!ctx->prof) return;
    const size_t need = 2 * (ctx->ev_pending.size() + 1);
    while (ctx->ev_pool.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ctx->ev_pool.push_back(e);
    }
    idx = (int)(2 * ctx->ev_pending.size());
    record(ctx->ev_pool[idx]);
  }
  ~Stage() {
    if (idx < 0) return;
    record(ctx->ev_pool[idx + 1]);
    ctx->ev_pending.push_back({id, idx});
  }
  // under stream capture an event must be recorded as an external node to be timed later
  void record(cudaEvent_t e) {
    if (ctx->capturing) cudaEventRecordWithFlags(e, ctx->st, cudaEventRecordExternal);
    else cudaEventRecord(e, ctx->st);
  }
};

// profiling mode 2: two spans that start together on the main stream (at the fork of the
// overlapped evaluation) and end on the stream given to span_end; returns the first span's
// event index or -1
void record_on(reaxff_ctx* ctx, cudaEvent_t e, cudaStream_t st) {
  if (ctx->capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}
int spans_begin(reaxff_ctx* ctx, int id0, int id1) {
  if (ctx->prof != 2) return -1;
  const size_t need = 2 * (ctx->ev_pending.size() + 2);
  while (ctx->ev_pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    ctx->ev_pool.push_back(e);
  }
  const int idx = (int)(2 * ctx->ev_pending.size());
  record_on(ctx, ctx->ev_pool[idx], ctx->st);
  record_on(ctx, ctx->ev_pool[idx + 2], ctx->st);
  ctx->ev_pending.push_back({id0, idx});
  ctx->ev_pending.push_back({id1, idx + 2});
  return idx;
}

void collect_profile(reaxff_ctx* ctx) {
  if (ctx->ev_pending.empty()) return;
  cudaStreamSynchronize(ctx->st);
  for (auto& p : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[p.second], ctx->ev_pool[p.second + 1]) == cudaSuccess) {
      ctx->stage_ms[p.first] += ms;
      ctx->stage_calls[p.first] += 1;
    }
  }
  ctx->ev_pending.clear();
}

int read_err(reaxff_ctx* ctx, int* flags) {
  CK(cudaMemcpyAsync(ctx->h_err_pinned, ctx->sys.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *flags = *ctx->h_err_pinned;
  return REAXFF_OK;
}

// capacities after an overflow (flags from the device)
void grow_caps(reaxff_ctx* ctx, int flags) {
  if (flags & ERR_CAP_FAR) ctx->cap_far = round_up(ctx->cap_far * 1.5, 32);
  if (flags & ERR_CAP_NEAR) ctx->cap_near = round_up(ctx->cap_near * 1.5, 32);
  if (flags & ERR_CAP_CAND) ctx->cap_cand = round_up(ctx->cap_cand * 1.5, 32);
  if (flags & ERR_CAP_BOND) ctx->cap_bond = round_up(ctx->cap_bond * 1.5, 8);
  if (flags & ERR_CAP_HB) ctx->cap_hb = round_up(ctx->cap_hb * 1.5, 32);
}

// checked: clear the flags, read them back after the build and regrow and retry on a
// capacity overflow (host synchronisation). Unchecked: launches only; the caller reads the
// flags later (the error word is not cleared, so earlier flags of a batch survive).
// drifted: the positions came from the fused drift kernel, which already wrote the float
// records and ran the skin test
// far_only (unchecked builds only): stop after the far and H-bond lists; the caller builds
// the bond list (bond_lists_impl) later, beside the QEq solve
void bond_lists_impl(reaxff_ctx* ctx, const rx::Launch& L) {
  if (ctx->fp64) rx::bond_list<double>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pd, ctx->Pd, ctx->use_skin);
  else rx::bond_list<float>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pf, ctx->Pd, ctx->use_skin);
  rx::bond_mirror(L, ctx->sys, ctx->bond);
  rx::bo_prime64(L, ctx->sys, ctx->bond, ctx->aq, ctx->Pd, ctx->n * ctx->bond.cap);
}

int build_lists_impl(reaxff_ctx* ctx, bool checked = true, bool drifted = false, bool far_only = false) {
  for (int attempt = 0; attempt < 3; ++attempt) {
    rx::Launch L = launch_of(ctx);
    if (checked) CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
    CK(cudaMemsetAsync(ctx->bond.ncanon, 0, sizeof(int), ctx->st));
    if (ctx->use_skin) {
      // Verlet-skin candidates (rebuilt on the device only when an atom moved > skin/2),
      // filtered exactly every step into the near/far rows
      { Stage st(ctx, 0);
        if (!drifted || attempt > 0) {
          rx::positions_f32(L, ctx->sys);
          rx::skin_check(L, ctx->sys, ctx->cand);
        }
        rx::cand_build(L, ctx->sys, ctx->cells, ctx->cand); }
      if (ctx->fp64) {
        { Stage st(ctx, 1); rx::cand_filter<double>(L, ctx->sys, ctx->cand, ctx->far, ctx->hb, ctx->Pd, ctx->far_margin, ctx->near_margin, ctx->hb_margin); }
        if (!far_only) { Stage st(ctx, 2); rx::bond_list<double>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pd, ctx->Pd, true); }
      } else {
        { Stage st(ctx, 1); rx::cand_filter<float>(L, ctx->sys, ctx->cand, ctx->far, ctx->hb, ctx->Pf, ctx->far_margin, ctx->near_margin, ctx->hb_margin); }
        if (!far_only) { Stage st(ctx, 2); rx::bond_list<float>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pf, ctx->Pd, true); }
      }
    } else {
    { Stage st(ctx, 0); rx::cells_build(L, ctx->sys, ctx->cells); }
    if (ctx->fp64) {
      { Stage st(ctx, 1); rx::far_list_split<double>(L, ctx->sys, ctx->cells, ctx->far, ctx->Pd, ctx->far_margin, ctx->near_margin); }
      if (!far_only) { Stage st(ctx, 2); rx::bond_list<double>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pd, ctx->Pd); }
    } else {
      { Stage st(ctx, 1); rx::far_list_split<float>(L, ctx->sys, ctx->cells, ctx->far, ctx->Pf, ctx->far_margin, ctx->near_margin); }
      if (!far_only) { Stage st(ctx, 2); rx::bond_list<float>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, ctx->Pf, ctx->Pd); }
    }
    }
    if (!far_only) {
      { Stage st(ctx, 2); rx::bond_mirror(L, ctx->sys, ctx->bond); }
      { Stage st(ctx, 3); rx::bo_prime64(L, ctx->sys, ctx->bond, ctx->aq, ctx->Pd, ctx->n * ctx->bond.cap); }
    }
    CK(cudaGetLastError());
    if (!checked) {
      ctx->lists_valid = true;
      return REAXFF_OK;
    }
    int flags = 0;
    int rc = read_err(ctx, &flags);
    if (rc) return rc;
    if (flags & ERR_NAN) return fail(ctx, REAXFF_E_NAN, "non-finite value while building lists");
    if (!(flags & (ERR_CAP_FAR | ERR_CAP_BOND | ERR_CAP_HB | ERR_CAP_NEAR | ERR_CAP_CAND))) {
      ctx->lists_valid = true;
      return REAXFF_OK;
    }
    if (attempt == 2) break;
    grow_caps(ctx, flags);
    int r2 = alloc_lists(ctx);
    if (r2) return r2;
    CK(cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st));   // candidates were reallocated
  }
  return fail(ctx, REAXFF_E_CAPACITY, "neighbour list capacity exceeded after regrow");
}

template <typename R> const DParams<R>* params_of(reaxff_ctx* ctx);
template <> const DParams<double>* params_of<double>(reaxff_ctx* ctx) { return ctx->Pd; }
template <> const DParams<float>* params_of<float>(reaxff_ctx* ctx) { return ctx->Pf; }

// side: on the second stream with the CG on 512 or 256 threads per SM (schedule), beside the
// charge-free terms (mixed path). The serial order with the stage timers on launches the CG
// in the shape the schedule gives it, so that its stage time is that launch's own.
int qeq_impl(reaxff_ctx* ctx, bool side = false) {
  rx::Launch L = launch_of(ctx);
  if (side) L.st = ctx->st2;
  const int ovl = (side || (ctx->prof == 1 && !ctx->fp64)) ? ctx->tune.qeq_overlap : 0;
  const int threads = ovl == 2 ? 256 : ovl == 1 ? 512 : 1024;
  const int layout = ovl >= 3 ? ovl - 2 : 0;
  const float* qhat = nullptr;
  if (ctx->ho.warm_start == REAXFF_WARM_MLP && ctx->mlp.alloc && ctx->mlp.ready) {
    // learned guess: descriptors of the current lists, tensor-core forward. Only a solve
    // without a usable solution history (the first one, or after a history reset, a re-sort
    // or a rolled-back call) takes it: with a history the extrapolated start is the better
    // one, so the kernels check the device history state and return at once
    Stage stg(ctx, 16);
    auto& M = ctx->mlp;
    rx::mlp_descriptors(L, ctx->sys, ctx->far, M.D, ctx->Q.hst);
    rx::mlp_infer(L, M.D, M.tiles, M.mean, M.inv, M.inf, M.y, ctx->sys.err, ctx->nsm, ctx->Q.hst);
    qhat = M.y;
  }
  if (ctx->Q.precond != REAXFF_PRECOND_JACOBI) {
    Stage stp(ctx, 17);
    rx::qeq_precond_build(L, ctx->sys, ctx->Q);
  }
  Stage stg(ctx, 4);
  int rc = ctx->fp64 ? rx::qeq_solve<double>(L, ctx->sys, ctx->far, ctx->Q, ctx->Pd, ctx->chi_t, ctx->eta_t,
                                             ctx->ho.qeq_tol, ctx->ho.qeq_max_iter, ctx->ho.warm_start, qhat)
                     : rx::qeq_solve<float>(L, ctx->sys, ctx->far, ctx->Q, ctx->Pf, ctx->chi_t, ctx->eta_t,
                                            ctx->ho.qeq_tol, ctx->ho.qeq_max_iter, ctx->ho.warm_start, qhat,
                                            threads, layout);
  if (rc) {
    cudaError_t e = cudaGetLastError();
    return fail(ctx, REAXFF_E_CUDA, "cooperative QEq launch failed: " + cuda_err_str(e));
  }
  return REAXFF_OK;
}

// Mixed path with the solve beside the charge-free terms. QEq (k_cg in the schedule's shape)
// and then the nonbonded kernel, the only charge-dependent term, run on the second stream;
// the bond list and bond orders (when bonds_pending), their corrections, atom terms, angles,
// torsions, H-bonds and the chain rule run on the main and third streams meanwhile. Neither
// side uses what the other writes: the solve writes charges (also into the fourth word of the
// packed position records, which the bond-list kernel loads with the positions but does not
// use), solutions and its own state; the terms read positions and bond data, write per-atom
// quantities and bond accumulators, and add forces, energies and the virial, like the
// nonbonded kernel, only through exact fixed-point atomics. So nothing races. The results
// agree with the serial order to within rounding: the CG thread count and rows per block
// change the order of the FP64 dot-product partials. Fork and join by events (graph edges
// under stream capture).
int forces_overlap(reaxff_ctx* ctx, bool bonds_pending) {
  rx::Launch L = launch_of(ctx);
  const DParams<float>* P = ctx->Pf;
  const int sp = spans_begin(ctx, STAGE_SOLVE_PATH, STAGE_TERMS_PATH);
  cudaEventRecord(ctx->ev_fork, ctx->st);
  cudaStreamWaitEvent(ctx->st2, ctx->ev_fork, 0);
  int rc = qeq_impl(ctx, true);
  if (rc) return rc;
  rx::Launch L2{ctx->st2, &ctx->launches, &ctx->tune};
  rx::nonbonded<float>(L2, ctx->sys, ctx->far, ctx->acc, P, ctx->mask);
  if (sp >= 0) record_on(ctx, ctx->ev_pool[sp + 1], ctx->st2);
  cudaEventRecord(ctx->ev_join, ctx->st2);
  if (bonds_pending) bond_lists_impl(ctx, L);      // the solve reads only the far list
  rx::bo_correct<float>(L, ctx->sys, ctx->bond, ctx->aq, P);
  rx::atom_terms<float>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
  // over/under-coordination with the bond energy, the S gather and the torsions on a third
  // stream beside the angle and H-bond kernels. The angle, torsion and H-bond kernels read
  // only the corrected bond orders and the atom quantities of the kernels above; the
  // over/under kernel's own outputs (dE/dS) are read by the S gather after it on the same
  // stream. Everything else they write (forces, energies, the virial, the dE/dBO and dE/dDelta
  // accumulators) is added through exact fixed-point atomics or owner-written per term, so
  // their order cannot matter; the chain rule, which reads the accumulators, waits for all
  cudaEventRecord(ctx->ev_fork3, ctx->st);
  cudaStreamWaitEvent(ctx->st3, ctx->ev_fork3, 0);
  rx::Launch L3{ctx->st3, &ctx->launches, &ctx->tune};
  rx::over_under_bond<float>(L3, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
  rx::s_gather<float>(L3, ctx->sys, ctx->bond, ctx->aq);
  rx::torsions<float>(L3, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
  cudaEventRecord(ctx->ev_join3, ctx->st3);
  rx::angles<float>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
  rx::hbonds<float>(L, ctx->sys, ctx->bond, ctx->hb, ctx->acc, P, ctx->mask);
  CK(cudaStreamWaitEvent(ctx->st, ctx->ev_join3, 0));
  rx::chain_rule<float>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc);
  if (sp >= 0) record_on(ctx, ctx->ev_pool[sp + 3], ctx->st);
  CK(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));
  return REAXFF_OK;
}

template <typename R> void terms_impl(reaxff_ctx* ctx) {
  rx::Launch L = launch_of(ctx);
  const DParams<R>* P = params_of<R>(ctx);
  { Stage st(ctx, 5); rx::bo_correct<R>(L, ctx->sys, ctx->bond, ctx->aq, P); }
  { Stage st(ctx, 6); rx::atom_terms<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); }
  { Stage st(ctx, 7); rx::over_under_bond<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); }
  { Stage st(ctx, 8); rx::s_gather<R>(L, ctx->sys, ctx->bond, ctx->aq); }
  if (sizeof(R) == 4 && ctx->prof != 1) {
    // the angle, torsion and H-bond terms (charge-independent) on the second stream beside the
    // nonbonded kernel: on the mixed path all four add their results through fixed-point
    // atomics only (exact, order-free) and read nothing another writes, so they commute;
    // fork and join by events (graph edges under stream capture). The stage timers keep the
    // serial order.
    cudaEventRecord(ctx->ev_fork, ctx->st);                 // errors surface at the caller's check
    cudaStreamWaitEvent(ctx->st2, ctx->ev_fork, 0);
    rx::Launch L2{ctx->st2, &ctx->launches, &ctx->tune};
    rx::angles<R>(L2, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
    rx::torsions<R>(L2, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask);
    rx::hbonds<R>(L2, ctx->sys, ctx->bond, ctx->hb, ctx->acc, P, ctx->mask);
    rx::nonbonded<R>(L, ctx->sys, ctx->far, ctx->acc, P, ctx->mask);
    cudaEventRecord(ctx->ev_join, ctx->st2);
    cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0);
  } else {
    { Stage st(ctx, 9); rx::angles<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); }
    { Stage st(ctx, 10); rx::torsions<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); }
    { Stage st(ctx, 11); rx::hbonds<R>(L, ctx->sys, ctx->bond, ctx->hb, ctx->acc, P, ctx->mask); }
    { Stage st(ctx, 12); rx::nonbonded<R>(L, ctx->sys, ctx->far, ctx->acc, P, ctx->mask); }
  }
  { Stage st(ctx, 13); rx::chain_rule<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc); }
}

int zero_accumulators(reaxff_ctx* ctx) {
  const size_t n = ctx->n, nb = n * ctx->bond.cap;
  CK(cudaMemsetAsync(ctx->sys.fx, 0, 3 * n * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->bond.cdbo, 0, nb * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->bond.cdbopi, 0, nb * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->bond.cdbopp, 0, nb * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->aq.cddelta, 0, n * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->aq.A, 0, n * sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(ctx->acc.e, 0, NTERMS * n * sizeof(double), ctx->st));
  CK(cudaMemsetAsync(ctx->acc.vir, 0, 6 * n * sizeof(double), ctx->st));
  CK(cudaMemsetAsync(ctx->acc.efx, 0, (NTERMS + 6) * n * sizeof(unsigned long long), ctx->st));   // efx and vfx
  return REAXFF_OK;
}

// lists -> (QEq) -> all terms -> chain rule; energies reduced into E_rep / vir_rep
int forces_impl(reaxff_ctx* ctx, bool solve_q, bool reduce = true, bool checked = true, bool drifted = false) {
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  const bool ovl = solve_q && !ctx->fp64 && ctx->prof != 1 && ctx->tune.qeq_overlap;
  // unchecked (MD steps): the bond list is built beside the solve; checked builds read the
  // capacity flags of every list before anything else runs
  const bool bonds_later = ovl && !checked;
  int rc = build_lists_impl(ctx, checked, drifted, bonds_later);
  if (rc) return rc;
  rc = zero_accumulators(ctx);
  if (rc) return rc;
  if (ovl) {
    rc = forces_overlap(ctx, bonds_later);
    if (rc) return rc;
  } else {
    if (solve_q) {
      rc = qeq_impl(ctx);
      if (rc) return rc;
    }
    if (ctx->fp64) terms_impl<double>(ctx);
    else terms_impl<float>(ctx);
  }
  if (reduce) {
    Stage st(ctx, 15);
    rx::reduce_energies(launch_of(ctx), ctx->sys, ctx->acc, ctx->mass_t, ctx->red, ctx->E_rep, ctx->vir_rep, ctx->ke_rep);
  }
  CK(cudaGetLastError());
  ctx->forces_valid = true;
  return REAXFF_OK;
}

// the status a set of device error flags stands for
int flags_status(reaxff_ctx* ctx, int flags, bool allow_nc) {
  if (flags & ERR_TIMEOUT) return fail(ctx, REAXFF_E_TIMEOUT, "a device-side wait hit its spin limit");
  if (flags & ERR_NAN) return fail(ctx, REAXFF_E_NAN, "non-finite or out-of-range value in forces/energies");
  if (flags & (ERR_CAP_FAR | ERR_CAP_BOND | ERR_CAP_HB | ERR_CAP_NEAR | ERR_CAP_CAND))
    return fail(ctx, REAXFF_E_CAPACITY, "list capacity exceeded");
  if ((flags & ERR_CG) && !allow_nc) return fail(ctx, REAXFF_E_NOT_CONVERGED, "QEq reached qeq_max_iter");
  if (flags & ERR_CG) {
    ctx->err = "QEq reached qeq_max_iter";
    return REAXFF_E_NOT_CONVERGED;
  }
  return REAXFF_OK;
}

int check_flags(reaxff_ctx* ctx, bool allow_nc) {
  int flags = 0;
  int rc = read_err(ctx, &flags);
  if (rc) return rc;
  return flags_status(ctx, flags, allow_nc);
}

// Initial-guess weights w[sys][m][k] of predictor `pred` (sys 0: s, 1: t; m newest solutions
// available, k = 0 the newest). Predictor 0, Lagrange: cubic through 4 points for s,
// quadratic through 3 for t. Predictors 1 and 2, least squares: the value at the next step
// of the polynomial of degree min(m' - 1, 3) fitted by least squares to the last m' =
// min(m, 6) or min(m, 8) solutions at equal steps (Lagrange up to 4 points, smoothing the
// solve-tolerance noise of the stored solutions beyond).
void extrap_weights(int pred, std::vector<double>& w) {
  const int H = rx::QEQ_HIST;
  w.assign(2 * (H + 1) * H, 0.0);
  for (int sys = 0; sys < 2; ++sys)
    for (int m = 1; m <= H; ++m) {
      double* o = w.data() + ((size_t)sys * (H + 1) + m) * H;
      int npt = std::min(m, pred == 1 ? 6 : H);
      int deg = std::min(npt - 1, 3);
      if (pred == 0) {
        deg = std::min(m - 1, sys == 0 ? 3 : 2);
        npt = deg + 1;
      }
      // normal equations (V^T V) c = e_0 for the fit to t_k = -(k + 1); w = V c
      double A[4][4] = {}, c[4] = {1.0, 0.0, 0.0, 0.0};
      const int D = deg + 1;
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b)
          for (int k = 0; k < npt; ++k) A[a][b] += std::pow(-(k + 1.0), a + b);
      for (int col = 0; col < D; ++col) {            // Gauss-Jordan (SPD, tiny)
        const double piv = A[col][col];
        for (int b = 0; b < D; ++b) A[col][b] /= piv;
        c[col] /= piv;
        for (int r = 0; r < D; ++r) {
          if (r == col) continue;
          const double f = A[r][col];
          for (int b = 0; b < D; ++b) A[r][b] -= f * A[col][b];
          c[r] -= f * c[col];
        }
      }
      for (int k = 0; k < npt; ++k) {
        double v = 0.0;
        for (int a = 0; a < D; ++a) v += std::pow(-(k + 1.0), a) * c[a];
        o[k] = v;
      }
    }
}

int validate(const reaxff_params* p, const reaxff_options* o, std::string& msg) {
  if (!p || !o) { msg = "null params/options"; return REAXFF_E_INVALID; }
  if (p->ntypes < 1 || p->ntypes > MAXT) { msg = "ntypes out of range"; return REAXFF_E_INVALID; }
  if (!(o->r_nb > 0 && o->r_bond > 0 && o->r_bond <= o->r_hb && o->r_hb <= o->r_nb)) {
    msg = "cutoffs must satisfy 0 < r_bond <= r_hb <= r_nb"; return REAXFF_E_INVALID;
  }
  if (!(o->bo_cut > 0 && o->qeq_tol > 0 && o->qeq_max_iter > 0)) { msg = "bo_cut, qeq_tol, qeq_max_iter must be > 0"; return REAXFF_E_INVALID; }
  if (o->precision != REAXFF_FP64 && o->precision != REAXFF_MIXED) { msg = "unknown precision"; return REAXFF_E_INVALID; }
  if (o->warm_start < 0 || o->warm_start > REAXFF_WARM_LAGRANGE) { msg = "unknown warm_start"; return REAXFF_E_INVALID; }
  if (!std::isfinite(o->skin) || o->skin > 5.0) { msg = "skin must be finite and <= 5 A"; return REAXFF_E_INVALID; }
  if (o->qeq_precond != REAXFF_PRECOND_JACOBI && o->qeq_precond != REAXFF_PRECOND_BLOCK32) {
    msg = "unknown qeq_precond"; return REAXFF_E_INVALID;
  }
  for (int a = 0; a < p->ntypes; ++a)
    if (!(p->mass[a] > 0 && p->eta[a] > 0)) { msg = "mass and eta must be > 0"; return REAXFF_E_INVALID; }
  return REAXFF_OK;
}

// ---- storage order ------------------------------------------------------------------------
// the caller's index of the atom stored at k
static inline int ext_of(const reaxff_ctx* ctx, int k) { return ctx->perm.empty() ? k : ctx->perm[(size_t)k]; }
// rows of w values: storage order -> the caller's order, and back
template <typename T> static void rows_to_caller(const reaxff_ctx* ctx, const T* src, T* dst, int w) {
  for (int k = 0; k < ctx->n; ++k)
    for (int c = 0; c < w; ++c) dst[(size_t)w * ext_of(ctx, k) + c] = src[(size_t)w * k + c];
}
template <typename T> static void rows_from_caller(const reaxff_ctx* ctx, const T* src, T* dst, int w) {
  for (int k = 0; k < ctx->n; ++k)
    for (int c = 0; c < w; ++c) dst[(size_t)w * k + c] = src[(size_t)w * ext_of(ctx, k) + c];
}
int mlp_tiles_upload(reaxff_ctx* ctx);

// Cell order of each replica's atoms from positions given in the caller's order (xyz rows):
// 5 A cells (at least one per axis), z-major, the caller's order within a cell. Switching to
// it rebuilds what depends on the order (types; the learned start's element tiles) and drops
// what cannot be carried over (solution history, bond-order averages, training snapshots).
static int apply_spatial_order(reaxff_ctx* ctx, const double* xs) {
  const int n = ctx->n;
  std::vector<int> perm(n);
  std::vector<std::pair<long long, int>> key;
  for (int r = 0; r < ctx->nrep; ++r) {
    const double* L = ctx->h_box.data() + 3 * r;
    int nc[3];
    for (int d = 0; d < 3; ++d) nc[d] = std::max(1, (int)std::floor(L[d] / 5.0));
    const int64_t a = ctx->h_rep_off[r], b = ctx->h_rep_off[r + 1];
    key.clear();
    for (int64_t i = a; i < b; ++i) {
      int c[3];
      for (int d = 0; d < 3; ++d) {
        double p = std::fmod(xs[3 * i + d], L[d]);
        if (p < 0) p += L[d];
        c[d] = std::min(nc[d] - 1, std::max(0, (int)std::floor(p / L[d] * nc[d])));
      }
      key.push_back({((long long)c[2] * nc[1] + c[1]) * nc[0] + c[0], (int)i});
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<long long, int>& u, const std::pair<long long, int>& v) { return u.first < v.first; });
    for (int64_t i = a; i < b; ++i) perm[i] = key[i - a].second;
  }
  ctx->perm.swap(perm);
  for (int k = 0; k < n; ++k) ctx->h_types[k] = ctx->h_types_ext[ctx->perm[k]];
  CK(cudaMemcpyAsync(ctx->type_d, ctx->h_types.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->Q.hst + 2, 0, sizeof(int), ctx->st));          // no usable solution history
  int rc = reaxff_bo_average_reset(ctx);
  if (rc) return rc;
  if (ctx->mlp.alloc) {
    ctx->mlp.count = 0;
    if ((rc = mlp_tiles_upload(ctx))) return rc;
  }
  CK(cudaStreamSynchronize(ctx->st));
  ctx->h_pos_valid = false;
  ctx->forces_valid = false;
  ctx->lists_valid = false;
  drop_graph(ctx);
  return REAXFF_OK;
}

}  // namespace

extern "C" {

int64_t reaxff_sizeof_params(void) { return (int64_t)sizeof(reaxff_params); }
int64_t reaxff_sizeof_options(void) { return (int64_t)sizeof(reaxff_options); }

int64_t reaxff_params_offset(const char* field) {
  if (!field) return -1;
#define OFS(f) if (!strcmp(field, #f)) return (int64_t)offsetof(reaxff_params, f);
  OFS(ntypes) OFS(hb) OFS(mass) OFS(val) OFS(vale) OFS(valboc) OFS(valang) OFS(p_lp2) OFS(p_ovun2)
  OFS(p_ovun5) OFS(p_val3) OFS(p_val5) OFS(chi) OFS(eta) OFS(gamma_t) OFS(r0s) OFS(r0p) OFS(r0pp)
  OFS(p_bo1) OFS(p_bo2) OFS(p_bo3) OFS(p_bo4) OFS(p_bo5) OFS(p_bo6) OFS(p_boc3) OFS(p_boc4) OFS(p_boc5)
  OFS(ovc) OFS(v13) OFS(De_s) OFS(De_p) OFS(De_pp) OFS(p_be1) OFS(p_be2) OFS(p_ovun1) OFS(vdw_D)
  OFS(vdw_rv) OFS(vdw_alpha) OFS(vdw_gw) OFS(gamma) OFS(th00) OFS(p_val1) OFS(p_val2) OFS(p_val4)
  OFS(p_val7) OFS(p_pen1) OFS(p_coa1) OFS(V1) OFS(V2) OFS(V3) OFS(p_tor1) OFS(p_cot1) OFS(r0hb)
  OFS(p_hb1) OFS(p_hb2) OFS(p_hb3) OFS(p_boc1) OFS(p_boc2) OFS(p_lp1) OFS(p_ovun3) OFS(p_ovun4)
  OFS(p_ovun6) OFS(p_ovun7) OFS(p_ovun8) OFS(p_val6) OFS(p_val8) OFS(p_val9) OFS(p_val10) OFS(p_pen2)
  OFS(p_pen3) OFS(p_pen4) OFS(p_coa2) OFS(p_coa3) OFS(p_coa4) OFS(p_tor2) OFS(p_tor3) OFS(p_tor4)
  OFS(p_cot2) OFS(p_vdW1) OFS(k_e)
#undef OFS
  return -1;
}

const char* reaxff_last_error(const reaxff_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int64_t reaxff_num_atoms(const reaxff_ctx* ctx) { return ctx ? ctx->n : 0; }
int32_t reaxff_num_replicas(const reaxff_ctx* ctx) { return ctx ? ctx->nrep : 0; }
int64_t reaxff_last_launch_count(const reaxff_ctx* ctx) { return ctx ? ctx->launches : 0; }

int reaxff_create_batch(const reaxff_params* params, int32_t nrep, const int64_t* rep_offsets,
                        const int32_t* types, const double* boxes, const reaxff_options* options,
                        reaxff_ctx** out) {
  if (!out) return REAXFF_E_INVALID;
  *out = nullptr;
  std::string msg;
  int v = validate(params, options, msg);
  if (v) return v;
  if (nrep < 1 || !rep_offsets || !types || !boxes || rep_offsets[0] != 0) return REAXFF_E_INVALID;
  for (int r = 0; r < nrep; ++r) {
    if (rep_offsets[r + 1] <= rep_offsets[r]) return REAXFF_E_INVALID;
    for (int d = 0; d < 3; ++d)
      if (!(boxes[3 * r + d] > options->r_nb)) return REAXFF_E_INVALID;
  }
  const int64_t n64 = rep_offsets[nrep];
  if (n64 > (int64_t)1 << 30) return REAXFF_E_INVALID;
  for (int64_t i = 0; i < n64; ++i)
    if (types[i] < 0 || types[i] >= params->ntypes) return REAXFF_E_INVALID;

  reaxff_ctx* ctx = new reaxff_ctx();
  ctx->n = (int)n64;
  ctx->nrep = nrep;
  ctx->hp = *params;
  ctx->ho = *options;
  ctx->fp64 = options->precision == REAXFF_FP64;
  ctx->mask = options->term_mask ? (unsigned)options->term_mask : 0x1fffu;
  ctx->h_rep_off.assign(rep_offsets, rep_offsets + nrep + 1);
  ctx->h_box.assign(boxes, boxes + 3 * nrep);
  ctx->h_types.assign(types, types + n64);
  ctx->h_types_ext.assign(types, types + n64);
  ctx->sort_on = options->spatial_sort != 0;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
  int coop = 0;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
  if (ce == cudaSuccess) {
    // the second stream at the highest priority: the persistent solve's blocks are placed
    // before those of the kernels beside it
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    ce = cudaStreamCreateWithPriority(&ctx->st2, cudaStreamNonBlocking, greatest);
  }
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&ctx->st3, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_fork3, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_join3, cudaEventDisableTiming);
  if (ce != cudaSuccess || !coop) {
    delete ctx;
    return REAXFF_E_CUDA;
  }
  const int n = ctx->n;
  // ---- capacities from the densest replica
  double rho = 0, lmax = 0;
  for (int r = 0; r < nrep; ++r) {
    double vol = boxes[3 * r] * boxes[3 * r + 1] * boxes[3 * r + 2];
    rho = std::max(rho, (double)(rep_offsets[r + 1] - rep_offsets[r]) / vol);
    for (int d = 0; d < 3; ++d) lmax = std::max(lmax, boxes[3 * r + d]);
  }
  const double margin = options->capacity_margin >= 1.0 ? options->capacity_margin : 1.35;
  const double sph = 4.0 / 3.0 * M_PI;
  ctx->cap_far = std::max(64, round_up(margin * sph * (std::pow(options->r_nb, 3) - std::pow(options->r_bond, 3)) * rho + 16, 32));
  ctx->cap_near = std::max(32, round_up(margin * sph * std::pow(options->r_bond, 3) * rho + 16, 32));
  // default 0.7 A: against 1.0 A, 8 % fewer candidates for the per-step filter outweigh
  // the more frequent rebuilds (petn32k 0.854 -> 0.844 ms per step, 1,039,360 atoms 22.0 ->
  // 21.8 ms, steady-state windows)
  ctx->skin = options->skin > 0.0 ? options->skin : 0.7;
  // candidates need every box edge above r_nb + skin (images beyond the nearest shifts stay
  // out of reach between rebuilds); smaller boxes run the cell stencil every step
  ctx->use_skin = !(options->skin < 0.0);
  for (int r = 0; r < nrep; ++r)
    for (int d = 0; d < 3; ++d)
      if (!(boxes[3 * r + d] > options->r_nb + ctx->skin)) ctx->use_skin = false;
  ctx->cap_cand = std::max(64, round_up(margin * sph * std::pow(options->r_nb + ctx->skin, 3) * rho + 16, 32));
  ctx->cap_bond = 24;
  ctx->cap_hb = std::max(32, round_up(margin * sph * std::pow(options->r_hb, 3) * rho + 16, 32));
  const double u = std::ldexp(1.0, -24);
  ctx->far_margin = (float)(32.0 * u * (lmax * options->r_nb + options->r_nb * options->r_nb));
  ctx->near_margin = (float)(32.0 * u * (lmax * options->r_bond + options->r_bond * options->r_bond));
  ctx->hb_margin = (float)(32.0 * u * (lmax * options->r_hb + options->r_hb * options->r_hb));
  {
    const double rc = options->r_nb + ctx->skin;
    ctx->cand.rc2 = (float)(rc * rc + 64.0 * u * (lmax * rc + rc * rc));
    ctx->cand.half_skin2 = 0.25 * ctx->skin * ctx->skin;
  }
  // ---- cells per replica: at least as wide as the largest distance the 27-cell stencil
  // must cover (r_nb, or r_nb + skin for the Verlet candidates)
  std::vector<int> nc(3 * nrep), cell_off(nrep + 1, 0);
  const double r_cell = ctx->use_skin ? options->r_nb + ctx->skin : options->r_nb;
  for (int r = 0; r < nrep; ++r) {
    int tot = 1;
    for (int d = 0; d < 3; ++d) {
      nc[3 * r + d] = std::max(1, (int)std::floor(boxes[3 * r + d] / r_cell));
      tot *= nc[3 * r + d];
    }
    cell_off[r + 1] = cell_off[r] + tot;
  }
  const int ncell = cell_off[nrep];
  // ---- fixed allocations
  DevBuf& B = ctx->fixed;
  ctx->Pd = B.alloc<DParams<double>>(1);
  ctx->Pf = B.alloc<DParams<float>>(1);
  Sys& s = ctx->sys;
  s.n = n;
  s.nrep = nrep;
  int* type_d = B.alloc<int>(n);
  int* rep_d = B.alloc<int>(n);
  double* box_d = B.alloc<double>(3 * nrep);
  int64_t* off_d = B.alloc<int64_t>(nrep + 1);
  float* boxh_d = B.alloc<float>(3 * nrep);
  float* boxl_d = B.alloc<float>(3 * nrep);
  s.type = type_d; s.rep = rep_d; s.box = box_d; s.rep_off = off_d; s.boxh = boxh_d; s.boxl = boxl_d;
  s.x = B.alloc<double>(n); s.y = B.alloc<double>(n); s.z = B.alloc<double>(n);
  s.xh = B.alloc<float>(n); s.yh = B.alloc<float>(n); s.zh = B.alloc<float>(n);
  s.xl = B.alloc<float>(n); s.yl = B.alloc<float>(n); s.zl = B.alloc<float>(n);
  s.vx = B.alloc<double>(n); s.vy = B.alloc<double>(n); s.vz = B.alloc<double>(n);
  unsigned long long* facc = B.alloc<unsigned long long>(3 * (size_t)n);
  s.fx = facc; s.fy = facc ? facc + n : nullptr; s.fz = facc ? facc + 2 * (size_t)n : nullptr;
  s.q = B.alloc<double>(n);
  s.qf = B.alloc<float>(n);
  s.ph = B.alloc<float4>(n);
  s.pl = B.alloc<float4>(n);
  s.err = B.alloc<int>(1);
  s.img = B.alloc<int>(3 * (size_t)n);
  s.xb = B.alloc<double>(3 * (size_t)n);
  s.rebuild = B.alloc<int>(1);
  Cells& c = ctx->cells;
  int* nc_d = B.alloc<int>(3 * nrep);
  int* coff_d = B.alloc<int>(nrep + 1);
  c.nc = nc_d; c.cell_off = coff_d; c.ncell_total = ncell;
  // candidate build: about four blocks per SM at least, each home cell's atoms shared by
  // this many blocks
  c.slices = std::max(1, std::min(16, (4 * ctx->nsm + ncell - 1) / std::max(ncell, 1)));
  c.count = B.alloc<int>(ncell); c.start = B.alloc<int>(ncell + 1); c.cursor = B.alloc<int>(ncell);
  c.atoms = B.alloc<int>(n); c.atom_cell = B.alloc<int>(n); c.tmp = B.alloc<int>(n);
  AtomQ& a = ctx->aq;
  double** aqf[] = {&a.dp, &a.dpboc, &a.sumbo, &a.delta, &a.dang, &a.nlp, &a.dnlp, &a.dlp, &a.dd,
                    &a.prodexp, &a.sbo2, &a.dsbo2, &a.sbo_fac, &a.cds};
  for (double** p : aqf) *p = B.alloc<double>(n);
  a.A = B.alloc<unsigned long long>(n);
  a.cddelta = B.alloc<unsigned long long>(n);
  a.sumbo_f = B.alloc<float>(n);
  a.dang_f = B.alloc<float>(n);
  for (float** p : {&a.delta_f, &a.sbo2_f, &a.dsbo2_f, &a.prodexp_f, &a.sbo_fac_f, &a.dnlp_f}) *p = B.alloc<float>(n);
  ctx->acc.e = B.alloc<double>((size_t)NTERMS * n);
  ctx->acc.vir = B.alloc<double>(6 * (size_t)n);
  ctx->acc.efx = B.alloc<unsigned long long>((NTERMS + 6) * (size_t)n);   // efx [NTERMS n], vfx [6n]
  ctx->acc.vfx = ctx->acc.efx + NTERMS * (size_t)n;
  ctx->F_out = B.alloc<double>(3 * (size_t)n);
  ctx->E_rep = B.alloc<double>(NTERMS * nrep);
  ctx->vir_rep = B.alloc<double>(6 * nrep);
  ctx->ke_rep = B.alloc<double>(nrep);
  ctx->chi_t = B.alloc<double>(MAXT);
  ctx->eta_t = B.alloc<double>(MAXT);
  ctx->mass_t = B.alloc<double>(2 * MAXT);          // masses, then their reciprocals
  double* ieta_d = B.alloc<double>(MAXT);
  ctx->Q.ieta = ieta_d;
  // ---- QEq state and chunking (chunks never straddle replicas)
  rx::QeqState& Q = ctx->Q;
  const int grid_all = rx::qeq_grid_size(ctx->nsm);
  Q.zg = B.alloc<double>(2 * (size_t)n);
  Q.hist_s = B.alloc<double>(2 * rx::QEQ_HIST * (size_t)n);   // s ring, then t ring
  Q.hist_t = Q.hist_s + rx::QEQ_HIST * (size_t)n;
  Q.wext = B.alloc<double>(rx::QEQ_NPRED * 2 * (rx::QEQ_HIST + 1) * rx::QEQ_HIST);
  Q.pred = B.alloc<int>(2 * nrep);
  Q.precond = options->qeq_precond;
  Q.Pf = ctx->Pf;
  // block-Jacobi blocks: 32 consecutive atoms of a replica (fewer at its end)
  std::vector<int> bjs, bjn;
  if (Q.precond == REAXFF_PRECOND_BLOCK32)
    for (int r = 0; r < nrep; ++r)
      for (int64_t i = rep_offsets[r]; i < rep_offsets[r + 1]; i += 32) {
        bjs.push_back((int)i);
        bjn.push_back((int)std::min<int64_t>(32, rep_offsets[r + 1] - i));
      }
  Q.bj_nblk = (int)bjs.size();
  Q.bj_start = Q.bj_nblk ? B.alloc<int>(Q.bj_nblk) : nullptr;
  Q.bj_size = Q.bj_nblk ? B.alloc<int>(Q.bj_nblk) : nullptr;
  Q.binv = Q.bj_nblk ? B.alloc<float>(32 * ((size_t)n + 32)) : nullptr;
  Q.ring_bytes = rx::qeq_ring_bytes(ctx->fp64);
  // launch shapes: chunks of about n / grid rows that never straddle replicas, and per block
  // its rows' state in shared memory when it fits
  std::vector<std::vector<int>> h_clo(rx::QEQ_NLAYOUT), h_crep(rx::QEQ_NLAYOUT), h_rchunk(rx::QEQ_NLAYOUT);
  size_t part_chunks = 0, scal_rows = 0, state_rows = 0;
  const size_t sc = (size_t)(nrep * rx::QEQ_SCAL_PER_REP + 4) * sizeof(double);
  for (int l = 0; l < rx::QEQ_NLAYOUT; ++l) {
    rx::QeqLayout& Y = Q.lay[l];
    Y.grid = std::max(1, grid_all * rx::QEQ_PART_NUM[l] / 8);
    int rows = std::max(8, (int)((n + Y.grid - 1) / Y.grid));
    if (Q.precond == REAXFF_PRECOND_BLOCK32) rows = round_up(rows, 32);   // chunks start on block boundaries
    std::vector<int>& clo = h_clo[l];
    std::vector<int>& crep = h_crep[l];
    std::vector<int>& rchunk = h_rchunk[l];
    rchunk.assign(nrep + 1, 0);
    for (int r = 0; r < nrep; ++r) {
      rchunk[r] = (int)crep.size();
      for (int64_t i = rep_offsets[r]; i < rep_offsets[r + 1]; i += rows) {
        clo.push_back((int)i);
        crep.push_back(r);
      }
    }
    rchunk[nrep] = (int)crep.size();
    Y.nchunk = (int)crep.size();
    clo.push_back(n);
    Y.chunk_lo = B.alloc<int>(clo.size());
    Y.chunk_rep = B.alloc<int>(crep.size());
    Y.rep_chunk = B.alloc<int>(nrep + 1);
    // rows per block (block b owns chunks b, b + grid, ...)
    std::vector<int> rowsb(Y.grid, 0);
    for (int c = 0; c < Y.nchunk; ++c) rowsb[c % Y.grid] += clo[c + 1] - clo[c];
    Y.rows_blk = *std::max_element(rowsb.begin(), rowsb.end());
    const size_t st = (size_t)rx::QEQ_NV_STATE * Y.rows_blk * sizeof(double);
    const size_t avail = (size_t)rx::QEQ_SMEM_MAX - Q.ring_bytes;
    Y.scal_smem = sc <= avail / 2;
    Y.state_smem = (Y.scal_smem ? sc : 0) + st <= avail;
    const size_t bjb = Q.precond == REAXFF_PRECOND_BLOCK32 ? (size_t)Y.rows_blk * 32 * sizeof(float) : 0;
    const size_t used = (Y.scal_smem ? sc : 0) + (Y.state_smem ? st : 0);
    Y.bj_smem = bjb > 0 && used + bjb <= avail;
    Y.smem_bytes = (int)(Q.ring_bytes + used + (Y.bj_smem ? bjb : 0));
    part_chunks = std::max(part_chunks, (size_t)Y.nchunk);
    if (!Y.scal_smem) scal_rows = std::max(scal_rows, (size_t)Y.grid);
    if (!Y.state_smem) state_rows = std::max(state_rows, (size_t)Y.grid * Y.rows_blk);
  }
  Q.part = B.alloc<double>(part_chunks * 2 * 8);
  Q.scal = scal_rows ? B.alloc<double>(scal_rows * (nrep * rx::QEQ_SCAL_PER_REP + 4)) : nullptr;
  Q.state = state_rows ? B.alloc<double>(state_rows * rx::QEQ_NV_STATE) : nullptr;
  // reduction chunks (<= RED_CHUNK atoms each, per replica)
  std::vector<int> rlo, rrep(nrep + 1, 0);
  for (int r = 0; r < nrep; ++r) {
    rrep[r] = (int)rlo.size();
    for (int64_t i = rep_offsets[r]; i < rep_offsets[r + 1]; i += rx::RED_CHUNK) rlo.push_back((int)i);
  }
  rrep[nrep] = (int)rlo.size();
  ctx->red.nchunk = (int)rlo.size();
  rlo.push_back(n);
  int* rlo_d = B.alloc<int>(rlo.size());
  int* rrep_d = B.alloc<int>(nrep + 1);
  std::vector<int> rcr(ctx->red.nchunk);                        // replica of each chunk
  for (int r = 0; r < nrep; ++r)
    for (int k = rrep[r]; k < rrep[r + 1]; ++k) rcr[k] = r;
  int* rcr_d = B.alloc<int>(std::max(1, ctx->red.nchunk));
  ctx->red.chunk_lo = rlo_d;
  ctx->red.chunk_rep = rcr_d;
  ctx->red.rep_chunk = rrep_d;
  ctx->red.part = B.alloc<double>((size_t)ctx->red.nchunk * 20);
  const size_t ndone = (size_t)nrep * 21 + 1;                   // (replica, quantity), replica, launch
  ctx->red.done = B.alloc<unsigned>(ndone);
  Q.iters = B.alloc<int>(2 * nrep);
  Q.bar = B.alloc<GridBar>(1);
  Q.hst = B.alloc<int>(4);
  Q.spmv_total = B.alloc<unsigned long long>(1);
  Q.mlp_used = B.alloc<int>(nrep);
  ctx->etot_buf = B.alloc<double>((size_t)ETOT_CHUNK * nrep);
  ctx->etot_idx = B.alloc<int>(1);
  ctx->snap = B.alloc<double>((6 + 2 * rx::QEQ_HIST) * (size_t)n);
  ctx->snap_i = B.alloc<int>(4);
  if (B.err != cudaSuccess) {
    std::string m = "allocation: " + cuda_err_str(B.err);
    B.free_all();
    cudaStreamDestroy(ctx->st);
    delete ctx;
    (void)m;
    return REAXFF_E_CUDA;
  }
  if (cudaMallocHost(&ctx->h_err_pinned, sizeof(int)) != cudaSuccess) {
    B.free_all();
    delete ctx;
    return REAXFF_E_CUDA;
  }
  // ---- uploads
  DParams<double> hd;
  DParams<float> hf;
  fill_params<double>(hd, *params, *options);
  fill_params<float>(hf, *params, *options);
  std::vector<int> rep_h(n);
  for (int r = 0; r < nrep; ++r)
    for (int64_t i = rep_offsets[r]; i < rep_offsets[r + 1]; ++i) rep_h[i] = r;
  std::vector<float> bh(3 * nrep), bl(3 * nrep);
  for (int k = 0; k < 3 * nrep; ++k) {
    bh[k] = (float)boxes[k];
    bl[k] = (float)(boxes[k] - (double)bh[k]);
  }
  double chi[MAXT], eta[MAXT], mass[MAXT], ieta[MAXT];
  for (int t = 0; t < MAXT; ++t) {
    chi[t] = params->chi[t]; eta[t] = params->eta[t]; mass[t] = params->mass[t];
    ieta[t] = params->eta[t] > 0 ? 1.0 / params->eta[t] : 0.0;
  }
  cudaError_t e = cudaSuccess;
#define UP(dst, src, bytes) if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice)
  UP(ctx->Pd, &hd, sizeof(hd));
  UP(ctx->Pf, &hf, sizeof(hf));
  UP(type_d, types, n * sizeof(int));
  ctx->type_d = type_d;
  UP(rep_d, rep_h.data(), n * sizeof(int));
  UP(box_d, boxes, 3 * nrep * sizeof(double));
  UP(off_d, rep_offsets, (nrep + 1) * sizeof(int64_t));
  UP(boxh_d, bh.data(), 3 * nrep * sizeof(float));
  UP(boxl_d, bl.data(), 3 * nrep * sizeof(float));
  UP(nc_d, nc.data(), 3 * nrep * sizeof(int));
  UP(coff_d, cell_off.data(), (nrep + 1) * sizeof(int));
  for (int l = 0; l < rx::QEQ_NLAYOUT; ++l) {
    UP(Q.lay[l].chunk_lo, h_clo[l].data(), h_clo[l].size() * sizeof(int));
    UP(Q.lay[l].chunk_rep, h_crep[l].data(), h_crep[l].size() * sizeof(int));
    UP(Q.lay[l].rep_chunk, h_rchunk[l].data(), (nrep + 1) * sizeof(int));
  }
  {
    std::vector<double> wx;
    for (int p = 0; p < rx::QEQ_NPRED; ++p) {
      std::vector<double> w1;
      extrap_weights(p, w1);
      wx.insert(wx.end(), w1.begin(), w1.end());
    }
    UP(Q.wext, wx.data(), wx.size() * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMemset(Q.pred, 0, 2 * nrep * sizeof(int));
  if (Q.bj_nblk) {
    UP(Q.bj_start, bjs.data(), bjs.size() * sizeof(int));
    UP(Q.bj_size, bjn.data(), bjn.size() * sizeof(int));
  }
  UP(rlo_d, rlo.data(), rlo.size() * sizeof(int));
  UP(rrep_d, rrep.data(), (nrep + 1) * sizeof(int));
  if (ctx->red.nchunk) UP(rcr_d, rcr.data(), rcr.size() * sizeof(int));
  UP(ctx->chi_t, chi, sizeof(chi));
  UP(ctx->eta_t, eta, sizeof(eta));
  double mass2[2 * MAXT];
  for (int t = 0; t < MAXT; ++t) {
    mass2[t] = mass[t];
    mass2[MAXT + t] = mass[t] > 0 ? 1.0 / mass[t] : 0.0;
  }
  UP(ctx->mass_t, mass2, sizeof(mass2));
  UP(ieta_d, ieta, sizeof(ieta));
#undef UP
  if (e == cudaSuccess) e = cudaMemset(s.vx, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s.vy, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s.vz, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s.q, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s.qf, 0, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s.ph, 0, n * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemset(s.pl, 0, n * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemset(s.img, 0, 3 * (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s.rebuild, 1, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->Q.hst, 0, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->Q.spmv_total, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(ctx->Q.mlp_used, 0, nrep * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->Q.bar, 0, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMemset(ctx->red.done, 0, ((size_t)nrep * 21 + 1) * sizeof(unsigned));
  if (e != cudaSuccess) {
    B.free_all();
    delete ctx;
    return REAXFF_E_CUDA;
  }
  if (alloc_lists(ctx)) {
    ctx->lists.free_all();
    B.free_all();
    delete ctx;
    return REAXFF_E_CUDA;
  }
  *out = ctx;
  return REAXFF_OK;
}

int reaxff_create(const reaxff_params* params, const int32_t* types, int64_t n, const double box[3],
                  const reaxff_options* options, reaxff_ctx** out) {
  if (n < 1 || !box) return REAXFF_E_INVALID;
  int64_t off[2] = {0, n};
  return reaxff_create_batch(params, 1, off, types, box, options, out);
}

void reaxff_destroy(reaxff_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  drop_graph(ctx);
  ctx->mlp.buf.free_all();
  ctx->mlp.data.free_all();
  ctx->spbuf.free_all();
  ctx->avgbuf.free_all();
  if (ctx->sp.h_changed) cudaFreeHost(ctx->sp.h_changed);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->Etot_dev) cudaFree(ctx->Etot_dev);
  if (ctx->h_etot) cudaFreeHost(ctx->h_etot);
  ctx->lists.free_all();
  ctx->fixed.free_all();
  if (ctx->h_err_pinned) cudaFreeHost(ctx->h_err_pinned);
  if (ctx->d_io) cudaFree(ctx->d_io);
  if (ctx->d_io_flag) cudaFree(ctx->d_io_flag);
  if (ctx->h_io_flag) cudaFreeHost(ctx->h_io_flag);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_fork3) cudaEventDestroy(ctx->ev_fork3);
  if (ctx->ev_join3) cudaEventDestroy(ctx->ev_join3);
  if (ctx->st3) cudaStreamDestroy(ctx->st3);
  if (ctx->st2) cudaStreamDestroy(ctx->st2);
  if (ctx->st) cudaStreamDestroy(ctx->st);
  delete ctx;
}

// ---- state I/O on the device (contexts whose atoms are stored in the caller's order)
namespace {
// caller's interleaved rows x[3n] (and v[3n], or zeros) -> SoA stage[6n] (x, y, z, vx, vy,
// vz) with each position wrapped into [0, L) of its replica exactly as the host path does it
// (fmod is exact; the same additions); flag bit 0: a non-finite position, bit 1: a wrapped
// position differs from the one the device holds (compared bit for bit; only when `cmp`)
__global__ void k_state_in(const double* __restrict__ x, const double* __restrict__ v, int n,
                           const int* __restrict__ rep, const double* __restrict__ box, const double* __restrict__ cx,
                           const double* __restrict__ cy, const double* __restrict__ cz, int cmp,
                           double* __restrict__ stage, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* L = box + 3 * rep[i];
  const double* cur[3] = {cx, cy, cz};
  int f = 0;
  for (int d = 0; d < 3; ++d) {
    double p = x[3 * (size_t)i + d];
    if (!(p >= 0.0 && p < L[d])) {
      if (!isfinite(p)) f |= 1;
      p = fmod(p, L[d]);
      if (p < 0) p += L[d];
      if (p >= L[d]) p -= L[d];
    }
    stage[d * (size_t)n + i] = p;
    stage[(3 + d) * (size_t)n + i] = v ? v[3 * (size_t)i + d] : 0.0;
    if (cmp && __double_as_longlong(p) != __double_as_longlong(cur[d][i])) f |= 2;
  }
  if (f) atomicOr(flag, f);
}
// staged rows (x, y, z, vx, vy, vz, n each) into the state
__global__ void k_state_commit(Sys s, const double* __restrict__ stage) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const size_t n = (size_t)s.n;
  s.x[i] = stage[i]; s.y[i] = stage[n + i]; s.z[i] = stage[2 * n + i];
  s.vx[i] = stage[3 * n + i]; s.vy[i] = stage[4 * n + i]; s.vz[i] = stage[5 * n + i];
}
// SoA state -> interleaved rows: x[3n], v[3n], q[n] at out, out + 3n, out + 6n
__global__ void k_state_out(Sys s, int want_x, int want_v, int want_q, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const size_t n3 = 3 * (size_t)s.n;
  if (want_x) {
    out[3 * (size_t)i] = s.x[i]; out[3 * (size_t)i + 1] = s.y[i]; out[3 * (size_t)i + 2] = s.z[i];
  }
  if (want_v) {
    out[n3 + 3 * (size_t)i] = s.vx[i]; out[n3 + 3 * (size_t)i + 1] = s.vy[i]; out[n3 + 3 * (size_t)i + 2] = s.vz[i];
  }
  if (want_q) out[2 * n3 + i] = s.q[i];
}
}  // namespace

static int io_buffers(reaxff_ctx* ctx) {
  if (!ctx->d_io) CK(cudaMalloc(&ctx->d_io, 13 * (size_t)ctx->n * sizeof(double)));
  if (!ctx->d_io_flag) CK(cudaMalloc(&ctx->d_io_flag, sizeof(int)));
  if (!ctx->h_io_flag) CK(cudaMallocHost(&ctx->h_io_flag, sizeof(int)));
  return REAXFF_OK;
}

// host rows -> device state with the unpacking, wrap, checks and comparison on the device:
// the host only issues the copies (one synchronisation, for the flags)
static int set_state_device_io(reaxff_ctx* ctx, const double* x, const double* v) {
  int rc;
  if ((rc = io_buffers(ctx))) return rc;
  const int n = ctx->n;
  const size_t n3 = 3 * (size_t)n;
  double* xin = ctx->d_io;
  double* vin = ctx->d_io + n3;
  double* stage = ctx->d_io + 2 * n3;
  CK(cudaMemcpyAsync(xin, x, n3 * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  if (v) CK(cudaMemcpyAsync(vin, v, n3 * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->d_io_flag, 0, sizeof(int), ctx->st));
  k_state_in<<<(n + 255) / 256, 256, 0, ctx->st>>>(xin, v ? vin : nullptr, n, ctx->sys.rep, ctx->sys.box, ctx->sys.x,
                                                   ctx->sys.y, ctx->sys.z, ctx->have_pos ? 1 : 0, stage,
                                                   ctx->d_io_flag);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_io_flag, ctx->d_io_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));                   // the caller's rows are consumed here
  const int flags = *ctx->h_io_flag;
  if (flags & 1) return fail(ctx, REAXFF_E_NAN, "non-finite position");
  // positions bit for bit those the device holds: forces, lists, candidates and image
  // counters stay valid (the copies below rewrite the same values)
  const bool same = ctx->have_pos && !(flags & 2);
  k_state_commit<<<(n + 255) / 256, 256, 0, ctx->st>>>(ctx->sys, stage);
  CK(cudaGetLastError());
  if (!same) {
    CK(cudaMemsetAsync(ctx->sys.img, 0, n3 * sizeof(int), ctx->st));
    CK(cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st));   // new positions: rebuild candidates
    ctx->have_pos = true;
    ctx->forces_valid = false;
    ctx->lists_valid = false;
  }
  ctx->h_pos_valid = false;                             // no host copy of the positions is kept
  return REAXFF_OK;
}

static int get_state_device_io(reaxff_ctx* ctx, double* x, double* v, double* q) {
  int rc;
  if ((rc = io_buffers(ctx))) return rc;
  const size_t n = ctx->n, n3 = 3 * n;
  k_state_out<<<(unsigned)((n + 255) / 256), 256, 0, ctx->st>>>(ctx->sys, x ? 1 : 0, v ? 1 : 0, q ? 1 : 0, ctx->d_io);
  CK(cudaGetLastError());
  if (x) CK(cudaMemcpyAsync(x, ctx->d_io, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (v) CK(cudaMemcpyAsync(v, ctx->d_io + n3, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (q) CK(cudaMemcpyAsync(q, ctx->d_io + 2 * n3, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return REAXFF_OK;
}

static int stage_buffer(reaxff_ctx* ctx) {
  if (!ctx->h_stage) CK(cudaMallocHost(&ctx->h_stage, 6 * (size_t)ctx->n * sizeof(double)));
  return REAXFF_OK;
}

static int set_state_common(reaxff_ctx* ctx, const double* x, const double* v, cudaMemcpyKind kind,
                            cudaStream_t user) {
  const int n = ctx->n;
  const size_t n3 = 3 * (size_t)n;
  int rc;
  if ((rc = stage_buffer(ctx))) return rc;
  // positions arrive interleaved xyz; de-interleave into SoA with wrap (pinned staging)
  std::vector<double> hx, hv;
  const double* xs = x;
  const double* vs = v;
  if (kind == cudaMemcpyDeviceToHost || kind == cudaMemcpyDeviceToDevice) {
    hx.resize(n3);
    CK(cudaMemcpyAsync(hx.data(), x, n3 * sizeof(double), cudaMemcpyDeviceToHost, user));
    if (v) {
      hv.resize(n3);
      CK(cudaMemcpyAsync(hv.data(), v, n3 * sizeof(double), cudaMemcpyDeviceToHost, user));
    }
    CK(cudaStreamSynchronize(user));
    xs = hx.data();
    vs = v ? hv.data() : nullptr;
  }
  if (ctx->sort_on && ctx->perm.empty()) {
    for (size_t e = 0; e < n3; ++e)
      if (!std::isfinite(xs[e])) return fail(ctx, REAXFF_E_NAN, "non-finite position");
    if ((rc = apply_spatial_order(ctx, xs))) return rc;
  }
  double* soa = ctx->h_stage;
  double* vsoa = ctx->h_stage + n3;
  for (int r = 0; r < ctx->nrep; ++r) {
    const double* L = ctx->h_box.data() + 3 * r;
    for (int64_t i = ctx->h_rep_off[r]; i < ctx->h_rep_off[r + 1]; ++i) {
      const int64_t e = ext_of(ctx, (int)i);             // the caller's row of stored atom i
      for (int d = 0; d < 3; ++d) {
        double p = xs[3 * e + d];
        if (!(p >= 0.0 && p < L[d])) {                   // outside the box (or not finite): wrap
          if (!std::isfinite(p)) return fail(ctx, REAXFF_E_NAN, "non-finite position");
          p = std::fmod(p, L[d]);
          if (p < 0) p += L[d];
          if (p >= L[d]) p -= L[d];
        }
        soa[d * (size_t)n + i] = p;
        vsoa[d * (size_t)n + i] = vs ? vs[3 * e + d] : 0.0;
      }
    }
  }
  // the same positions as the device holds (bit for bit): forces, lists, candidates and
  // image counters stay valid (the copy below rewrites the same values)
  const bool same = ctx->have_pos && ctx->h_pos_valid &&
                    std::memcmp(soa, ctx->h_pos.data(), n3 * sizeof(double)) == 0;
  CK(cudaMemcpyAsync(ctx->sys.x, soa, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->sys.y, soa + n, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->sys.z, soa + 2 * (size_t)n, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->sys.vx, vsoa, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->sys.vy, vsoa + n, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->sys.vz, vsoa + 2 * (size_t)n, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  if (!same) {
    CK(cudaMemsetAsync(ctx->sys.img, 0, n3 * sizeof(int), ctx->st));
    CK(cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st));   // new positions: rebuild candidates
    ctx->h_pos.assign(soa, soa + n3);
    ctx->h_pos_valid = true;
  }
  CK(cudaStreamSynchronize(ctx->st));                   // the staging buffer is reused next call
  if (!same) {
    ctx->have_pos = true;
    ctx->forces_valid = false;
    ctx->lists_valid = false;
  }
  return REAXFF_OK;
}

int reaxff_set_state(reaxff_ctx* ctx, const double* x, const double* v) {
  if (!ctx || !x) return REAXFF_E_INVALID;
  if (!ctx->sort_on) return set_state_device_io(ctx, x, v);
  return set_state_common(ctx, x, v, cudaMemcpyHostToHost, ctx->st);
}

int reaxff_resort(reaxff_ctx* ctx) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->sort_on) return REAXFF_OK;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  const size_t n3 = 3 * (size_t)ctx->n;
  std::vector<double> x(n3), v(n3);
  int rc;
  if ((rc = reaxff_get_state(ctx, x.data(), v.data(), nullptr))) return rc;
  if ((rc = apply_spatial_order(ctx, x.data()))) return rc;
  return set_state_common(ctx, x.data(), v.data(), cudaMemcpyHostToHost, ctx->st);
}

int reaxff_set_state_dev(reaxff_ctx* ctx, const double* x_dev, const double* v_dev, void* stream) {
  if (!ctx || !x_dev) return REAXFF_E_INVALID;
  return set_state_common(ctx, x_dev, v_dev, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
}

// three device arrays (SoA) into interleaved host out[3n], through the pinned staging buffer;
// positions (a == sys.x) are also kept as the host copy of the device positions
static int get_soa3(reaxff_ctx* ctx, const double* a, const double* b, const double* c, double* out) {
  const int n = ctx->n;
  int rc;
  if ((rc = stage_buffer(ctx))) return rc;
  double* t = ctx->h_stage;
  CK(cudaMemcpyAsync(t, a, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(t + n, b, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(t + 2 * (size_t)n, c, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) out[3 * (size_t)ext_of(ctx, i) + d] = t[d * (size_t)n + i];
  if (a == ctx->sys.x) {
    ctx->h_pos.assign(t, t + 3 * (size_t)n);
    ctx->h_pos_valid = true;
  }
  return REAXFF_OK;
}

int reaxff_get_state(reaxff_ctx* ctx, double* x, double* v, double* q) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  if (ctx->perm.empty()) return get_state_device_io(ctx, x, v, q);
  int rc;
  if (x && (rc = get_soa3(ctx, ctx->sys.x, ctx->sys.y, ctx->sys.z, x))) return rc;
  if (v && (rc = get_soa3(ctx, ctx->sys.vx, ctx->sys.vy, ctx->sys.vz, v))) return rc;
  if (q) {
    std::vector<double> t(ctx->n);
    CK(cudaMemcpyAsync(t.data(), ctx->sys.q, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    rows_to_caller(ctx, t.data(), q, 1);
  }
  return REAXFF_OK;
}

int reaxff_get_state_dev(reaxff_ctx* ctx, double* x_dev, double* v_dev, double* q_dev, void* stream) {
  if (!ctx) return REAXFF_E_INVALID;
  std::vector<double> tmp(3 * (size_t)ctx->n);
  int rc;
  if (x_dev) {
    if ((rc = get_soa3(ctx, ctx->sys.x, ctx->sys.y, ctx->sys.z, tmp.data()))) return rc;
    CK(cudaMemcpyAsync(x_dev, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
  }
  if (v_dev) {
    if ((rc = get_soa3(ctx, ctx->sys.vx, ctx->sys.vy, ctx->sys.vz, tmp.data()))) return rc;
    CK(cudaMemcpyAsync(v_dev, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
  }
  if (q_dev) {
    std::vector<double> t(ctx->n), u(ctx->n);
    CK(cudaMemcpyAsync(t.data(), ctx->sys.q, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    rows_to_caller(ctx, t.data(), u.data(), 1);
    CK(cudaMemcpyAsync(q_dev, u.data(), ctx->n * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
  }
  return REAXFF_OK;
}

int reaxff_build_lists(reaxff_ctx* ctx) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  return build_lists_impl(ctx);
}

int reaxff_get_lists(reaxff_ctx* ctx, int32_t which, int64_t capacity, int64_t* count, int32_t* i_out,
                     int32_t* j_out, int8_t* shift) {
  if (!ctx || !count) return REAXFF_E_INVALID;
  if (!ctx->lists_valid) return fail(ctx, REAXFF_E_STATE, "lists not built");
  const int n = ctx->n;
  struct Part { int cap; const int* cnt; const int* j; const uint8_t* s; };
  std::vector<Part> parts;
  if (which == REAXFF_LIST_FAR) {
    parts.push_back({ctx->far.capn, ctx->far.cntn, ctx->far.jn, ctx->far.sn});
    parts.push_back({ctx->far.cap, ctx->far.cnt, ctx->far.j, ctx->far.s});
  } else if (which == REAXFF_LIST_BOND) {
    parts.push_back({ctx->bond.cap, ctx->bond.cnt, ctx->bond.j, ctx->bond.s});
  } else if (which == REAXFF_LIST_HBOND) {
    parts.push_back({ctx->hb.cap, ctx->hb.cnt, ctx->hb.j, ctx->hb.s});
  } else {
    return fail(ctx, REAXFF_E_INVALID, "unknown list");
  }
  std::vector<std::vector<int>> cnts(parts.size(), std::vector<int>(n));
  int64_t tot = 0;
  for (size_t p = 0; p < parts.size(); ++p) {
    CK(cudaMemcpyAsync(cnts[p].data(), parts[p].cnt, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int i = 0; i < n; ++i) tot += cnts[p][i];
  }
  *count = tot;
  if (capacity == 0 && !i_out) return REAXFF_OK;
  if (capacity < tot || !i_out || !j_out || !shift) return fail(ctx, REAXFF_E_INVALID, "output capacity too small");
  std::vector<std::vector<int>> jj(parts.size());
  std::vector<std::vector<uint8_t>> ss(parts.size());
  for (size_t p = 0; p < parts.size(); ++p) {
    jj[p].resize((size_t)n * parts[p].cap);
    ss[p].resize((size_t)n * parts[p].cap);
    CK(cudaMemcpyAsync(jj[p].data(), parts[p].j, jj[p].size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ss[p].data(), parts[p].s, ss[p].size(), cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  int64_t k = 0;
  for (int i = 0; i < n; ++i)
    for (size_t p = 0; p < parts.size(); ++p)
      for (int m = 0; m < cnts[p][i]; ++m) {
        const size_t e = (size_t)i * parts[p].cap + m;
        i_out[k] = ext_of(ctx, i);
        j_out[k] = ext_of(ctx, jj[p][e]);
        const int c = ss[p][e];
        shift[3 * k + 0] = (int8_t)(c / 9 - 1);
        shift[3 * k + 1] = (int8_t)((c / 3) % 3 - 1);
        shift[3 * k + 2] = (int8_t)(c % 3 - 1);
        ++k;
      }
  return REAXFF_OK;
}

int reaxff_get_bond_orders(reaxff_ctx* ctx, int64_t capacity, int64_t* count, double* bo_prime, double* bo,
                           double* bo_pi, double* bo_pipi) {
  if (!ctx || !count) return REAXFF_E_INVALID;
  if (!ctx->forces_valid) return fail(ctx, REAXFF_E_STATE, "call reaxff_forces first");
  const int n = ctx->n, cap = ctx->bond.cap;
  std::vector<int> cnt(n);
  CK(cudaMemcpyAsync(cnt.data(), ctx->bond.cnt, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  int64_t tot = 0;
  for (int i = 0; i < n; ++i) tot += cnt[i];
  *count = tot;
  if (capacity == 0 && !bo) return REAXFF_OK;
  if (capacity < tot) return fail(ctx, REAXFF_E_INVALID, "output capacity too small");
  void* src[4] = {ctx->bond.bop, ctx->bond.bo, ctx->bond.bo_pi, ctx->bond.bo_pp};
  double* dst[4] = {bo_prime, bo, bo_pi, bo_pipi};
  for (int f = 0; f < 4; ++f) {
    if (!dst[f]) continue;
    const bool dbl = ctx->fp64 || f == 0;          // BO' is FP64 in both modes
    std::vector<char> buf((size_t)n * cap * (dbl ? 8 : 4));
    CK(cudaMemcpyAsync(buf.data(), src[f], buf.size(), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    int64_t k = 0;
    for (int i = 0; i < n; ++i)
      for (int m = 0; m < cnt[i]; ++m) {
        const size_t e = (size_t)i * cap + m;
        dst[f][k++] = dbl ? ((double*)buf.data())[e] : (double)((float*)buf.data())[e];
      }
  }
  return REAXFF_OK;
}

int reaxff_qeq(reaxff_ctx* ctx, double* q_out, int32_t* iters_s, int32_t* iters_t) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  int rc = build_lists_impl(ctx);
  if (rc) return rc;
  rc = qeq_impl(ctx);
  if (rc) return rc;
  int frc = check_flags(ctx, true);
  if (frc && frc != REAXFF_E_NOT_CONVERGED) return frc;
  std::vector<int> it(2 * ctx->nrep);
  std::vector<double> qs(q_out ? ctx->n : 0);
  CK(cudaMemcpyAsync(it.data(), ctx->Q.iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (q_out) CK(cudaMemcpyAsync(qs.data(), ctx->sys.q, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (q_out) rows_to_caller(ctx, qs.data(), q_out, 1);
  for (int r = 0; r < ctx->nrep; ++r) {
    if (iters_s) iters_s[r] = it[2 * r];
    if (iters_t) iters_t[r] = it[2 * r + 1];
  }
  return frc;
}

static int copy_outputs(reaxff_ctx* ctx, double* F, double* E, double* virial) {
  std::vector<double> Fs(F && !ctx->perm.empty() ? 3 * (size_t)ctx->n : 0);
  if (F) {
    rx::finalize_forces(launch_of(ctx), ctx->sys, ctx->F_out);
    CK(cudaMemcpyAsync(Fs.empty() ? F : Fs.data(), ctx->F_out, 3 * (size_t)ctx->n * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->st));
  }
  if (E) CK(cudaMemcpyAsync(E, ctx->E_rep, NTERMS * ctx->nrep * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (virial) CK(cudaMemcpyAsync(virial, ctx->vir_rep, 6 * ctx->nrep * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (!Fs.empty()) rows_to_caller(ctx, Fs.data(), F, 3);
  return REAXFF_OK;
}

int reaxff_forces(reaxff_ctx* ctx, double* F, double* E, double* virial) {
  if (!ctx) return REAXFF_E_INVALID;
  int rc = forces_impl(ctx, true);
  if (rc) return rc;
  int frc = check_flags(ctx, true);
  if (frc && frc != REAXFF_E_NOT_CONVERGED) return frc;
  rc = copy_outputs(ctx, F, E, virial);
  return rc ? rc : frc;
}

int reaxff_forces_fixed_q(reaxff_ctx* ctx, const double* q, double* F, double* E, double* virial) {
  if (!ctx || !q) return REAXFF_E_INVALID;
  std::vector<double> qs(ctx->n);
  rows_from_caller(ctx, q, qs.data(), 1);
  CK(cudaMemcpyAsync(ctx->sys.q, qs.data(), ctx->n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  rx::charges_to_f32(launch_of(ctx), ctx->sys);
  int rc = forces_impl(ctx, false);
  if (rc) return rc;
  rc = check_flags(ctx, false);
  if (rc) return rc;
  return copy_outputs(ctx, F, E, virial);
}

// one velocity-Verlet step's launches (forces of the current positions are valid on entry);
// the total energy per replica goes to Etot_out (at *etot_idx when given)
static int step_once(reaxff_ctx* ctx, double dt, bool checked, double* Etot_out, int* etot_idx) {
  rx::Launch L = launch_of(ctx);
  { Stage sg(ctx, 14); rx::verlet_kick_drift(L, ctx->sys, ctx->mass_t, dt, 1, ctx->use_skin ? &ctx->cand : nullptr); }
  int rc = forces_impl(ctx, true, false, checked, ctx->use_skin);
  if (rc) return rc;
  { Stage sg(ctx, 14); rx::verlet_kick_drift(L, ctx->sys, ctx->mass_t, dt, 0); }
  Stage sg(ctx, 15);
  rx::reduce_energies(L, ctx->sys, ctx->acc, ctx->mass_t, ctx->red, ctx->E_rep, ctx->vir_rep, ctx->ke_rep, Etot_out,
                      etot_idx);
  return REAXFF_OK;
}

// capture one unchecked step into a CUDA graph; false when capture is not available
static bool capture_step(reaxff_ctx* ctx, double dt) {
  drop_graph(ctx);
  collect_profile(ctx);
  if (ctx->prof)
    while (ctx->ev_pool.size() < 64) {                 // no event creation during capture
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return false;
      ctx->ev_pool.push_back(e);
    }
  const int64_t l0 = ctx->launches;
  if (cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->capturing = true;
  const int rc = step_once(ctx, dt, false, ctx->etot_buf, ctx->etot_idx);
  ctx->capturing = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
  if (rc == REAXFF_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&ctx->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
  if (g) cudaGraphDestroy(g);
  const bool ok = rc == REAXFF_OK && e == cudaSuccess && ctx->gexec;
  if (!ok) {
    cudaGetLastError();
    ctx->gexec = nullptr;
    ctx->ev_pending.clear();
    ctx->launches = l0;
    return false;
  }
  ctx->g_launches = ctx->launches - l0;
  ctx->launches = l0;
  ctx->g_events.swap(ctx->ev_pending);
  ctx->ev_pending.clear();
  ctx->g_dt = dt;
  ctx->g_prof = ctx->prof;
  return true;
}

// stage times of the last graph replay (its event-record nodes)
static void collect_graph_profile(reaxff_ctx* ctx) {
  cudaStreamSynchronize(ctx->st);
  for (auto& p : ctx->g_events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[p.second], ctx->ev_pool[p.second + 1]) == cudaSuccess) {
      ctx->stage_ms[p.first] += ms;
      ctx->stage_calls[p.first] += 1;
    }
  }
}

// the steps of one call without host synchronisation; returns the device flags. With
// Etot_host (pinned), the energies are copied there before the flags are read, so that the
// one synchronisation of the flag read covers both
static int run_unchecked(reaxff_ctx* ctx, int nsteps, double dt, double* Etot_dev, int* flags,
                         double* Etot_host = nullptr) {
  rx::Launch L = launch_of(ctx);
  rx::snapshot(L, ctx->sys, ctx->Q.hist_s, 2 * rx::QEQ_HIST * ctx->n, ctx->Q.hst, ctx->snap, ctx->snap_i, 0);
  CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
  for (int c0 = 0; c0 < nsteps; c0 += ETOT_CHUNK) {
    const int len = std::min(ETOT_CHUNK, nsteps - c0);
    CK(cudaMemsetAsync(ctx->etot_idx, 0, sizeof(int), ctx->st));
    for (int k = 0; k < len; ++k) {
      if (ctx->graph_ok && (!ctx->gexec || ctx->g_dt != dt || ctx->g_prof != ctx->prof))
        ctx->graph_ok = capture_step(ctx, dt);
      if (ctx->graph_ok) {
        CK(cudaGraphLaunch(ctx->gexec, ctx->st));
        ctx->launches += ctx->g_launches;
        if (ctx->prof) collect_graph_profile(ctx);
      } else {
        int rc = step_once(ctx, dt, false, ctx->etot_buf, ctx->etot_idx);
        if (rc) return rc;
      }
    }
    if (Etot_dev)
      CK(cudaMemcpyAsync(Etot_dev + (size_t)c0 * ctx->nrep, ctx->etot_buf, (size_t)len * ctx->nrep * sizeof(double),
                         cudaMemcpyDeviceToDevice, ctx->st));
  }
  if (Etot_dev && Etot_host)
    CK(cudaMemcpyAsync(Etot_host, Etot_dev, (size_t)nsteps * ctx->nrep * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->st));
  CK(cudaGetLastError());
  return read_err(ctx, flags);
}

// Etot_host (pinned, or null): *staged is set when the energies of the call already sit there
static int step_impl(reaxff_ctx* ctx, int nsteps, double dt, double* Etot_dev, double* Etot_host = nullptr,
                     bool* staged = nullptr) {
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  ctx->launches = 0;
  if (nsteps > 0) ctx->h_pos_valid = false;               // the atoms move
  int rc;
  if (!ctx->forces_valid) {
    if ((rc = forces_impl(ctx, true))) return rc;
  }
  if (nsteps > 0) {
    int flags = 0;
    if ((rc = run_unchecked(ctx, nsteps, dt, Etot_dev, &flags, Etot_host))) return rc;
    const int cap = ERR_CAP_FAR | ERR_CAP_BOND | ERR_CAP_HB | ERR_CAP_NEAR | ERR_CAP_CAND;
    if (!(flags & cap) || (flags & (ERR_NAN | ERR_TIMEOUT))) {
      rc = flags_status(ctx, flags, false);               // the flags were read after the last step
      collect_profile(ctx);
      if (staged) *staged = Etot_dev && Etot_host;
      return rc;
    }
    // a list overflowed during the call: restore its starting state, regrow, redo it checked
    rx::Launch L = launch_of(ctx);
    rx::snapshot(L, ctx->sys, ctx->Q.hist_s, 2 * rx::QEQ_HIST * ctx->n, ctx->Q.hst, ctx->snap, ctx->snap_i, 1);
    CK(cudaMemsetAsync(ctx->sys.img, 0, 3 * (size_t)ctx->n * sizeof(int), ctx->st));
    CK(cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st));
    grow_caps(ctx, flags);
    if ((rc = alloc_lists(ctx))) return rc;
    CK(cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st));
    ctx->forces_valid = false;
    if ((rc = forces_impl(ctx, true))) return rc;
  }
  for (int st = 0; st < nsteps; ++st) {
    if ((rc = step_once(ctx, dt, true, Etot_dev ? Etot_dev + (size_t)st * ctx->nrep : ctx->etot_buf, nullptr)))
      return rc;
  }
  CK(cudaGetLastError());
  rc = check_flags(ctx, false);
  collect_profile(ctx);
  return rc;
}

int reaxff_step(reaxff_ctx* ctx, int32_t nsteps, double dt_fs, double* E_tot) {
  if (!ctx || nsteps < 0 || !(dt_fs > 0)) return REAXFF_E_INVALID;
  double* dev = nullptr;
  const size_t ebytes = (size_t)nsteps * ctx->nrep * sizeof(double);
  if (E_tot && nsteps > 0) {
    if (ctx->Etot_cap < nsteps * ctx->nrep) {
      if (ctx->Etot_dev) cudaFree(ctx->Etot_dev);
      if (ctx->h_etot) cudaFreeHost(ctx->h_etot);
      ctx->Etot_dev = nullptr;
      ctx->h_etot = nullptr;
      ctx->Etot_cap = 0;
      CK(cudaMalloc(&ctx->Etot_dev, ebytes));
      CK(cudaMallocHost(&ctx->h_etot, ebytes));
      ctx->Etot_cap = nsteps * ctx->nrep;
    }
    dev = ctx->Etot_dev;
  }
  // the energies come back through a pinned buffer, in the synchronisation that reads the
  // call's error flags
  bool staged = false;
  int rc = step_impl(ctx, nsteps, dt_fs, dev, dev ? ctx->h_etot : nullptr, &staged);
  if (rc) return rc;
  if (E_tot && nsteps > 0) {
    if (!staged) {
      CK(cudaMemcpyAsync(ctx->h_etot, dev, ebytes, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    std::memcpy(E_tot, ctx->h_etot, ebytes);
  }
  return REAXFF_OK;
}

int reaxff_last_qeq_iters(reaxff_ctx* ctx, int32_t* iters_s, int32_t* iters_t) {
  if (!ctx) return REAXFF_E_INVALID;
  std::vector<int> it(2 * ctx->nrep);
  CK(cudaMemcpyAsync(it.data(), ctx->Q.iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int r = 0; r < ctx->nrep; ++r) {
    if (iters_s) iters_s[r] = it[2 * r];
    if (iters_t) iters_t[r] = it[2 * r + 1];
  }
  return REAXFF_OK;
}

int reaxff_qeq_warm_choice(reaxff_ctx* ctx, int32_t* mlp_used) {
  if (!ctx || !mlp_used) return REAXFF_E_INVALID;
  CK(cudaMemcpyAsync(mlp_used, ctx->Q.mlp_used, ctx->nrep * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return REAXFF_OK;
}

int64_t reaxff_qeq_spmv_total(reaxff_ctx* ctx) {
  if (!ctx) return -1;
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, ctx->Q.spmv_total, sizeof(v), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return -1;
  return (int64_t)v;
}

int reaxff_set_wait_limit(reaxff_ctx* ctx, int64_t cycles) {
  if (!ctx) return REAXFF_E_INVALID;
  ctx->Q.bar_limit = cycles > 0 ? (long long)cycles : 0;
  drop_graph(ctx);                                   // captured launches carry the old limit
  return REAXFF_OK;
}

void reaxff_reset_qeq_history(reaxff_ctx* ctx) {
  if (ctx) cudaMemsetAsync(ctx->Q.hst + 2, 0, sizeof(int), ctx->st);   // no usable history
}

void reaxff_profile_enable(reaxff_ctx* ctx, int32_t on) {
  if (!ctx) return;
  ctx->prof = on == 2 ? 2 : on != 0 ? 1 : 0;
  for (int s = 0; s < 32; ++s) { ctx->stage_ms[s] = 0; ctx->stage_calls[s] = 0; }
}

int32_t reaxff_profile_read(reaxff_ctx* ctx, int32_t nstage, double* ms, int64_t* calls) {
  if (!ctx) return 0;
  collect_profile(ctx);
  for (int s = 0; s < nstage && s < NSTAGES; ++s) {
    if (ms) ms[s] = ctx->stage_ms[s];
    if (calls) calls[s] = ctx->stage_calls[s];
  }
  return NSTAGES;
}

const char* reaxff_stage_name(int32_t stage) {
  return (stage >= 0 && stage < NSTAGES) ? STAGE_NAMES[stage] : "";
}

int reaxff_step_dev(reaxff_ctx* ctx, int32_t nsteps, double dt_fs, double* E_tot_dev, void* stream) {
  if (!ctx || nsteps < 0 || !(dt_fs > 0)) return REAXFF_E_INVALID;
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, (cudaStream_t)stream));
  CK(cudaStreamWaitEvent(ctx->st, ev, 0));
  int rc = step_impl(ctx, nsteps, dt_fs, E_tot_dev);
  CK(cudaEventRecord(ev, ctx->st));
  CK(cudaStreamWaitEvent((cudaStream_t)stream, ev, 0));
  cudaEventDestroy(ev);
  return rc;
}

}  // extern "C"

// ------------------------------------------------------------------ learned warm start
namespace {
// element tiles over m samples with the given elements (host side: counting sort, stable)
void mlp_tiles_host(const std::vector<int>& types, std::vector<int>& perm, std::vector<int>& tile_type,
                    std::vector<int>& rows_off, int off[5]) {
  const int m = (int)types.size();
  perm.clear(); tile_type.clear(); rows_off.clear();
  for (int t = 0; t < rx::MLP_NT; ++t) {
    off[t] = (int)perm.size();
    for (int i = 0; i < m; ++i)
      if (types[i] == t) perm.push_back(i);
    for (int r = off[t]; r < (int)perm.size(); r += 128) {
      tile_type.push_back(t);
      rows_off.push_back(r);
    }
  }
  off[rx::MLP_NT] = (int)perm.size();
  rows_off.push_back((int)perm.size());
}

// splitmix64 -> uniform (0, 1)
double u01(uint64_t& st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) + 0.5) / 9007199254740992.0;
}

// element tiles and per-atom elements of the current storage order
int mlp_tiles_upload(reaxff_ctx* ctx) {
  auto& M = ctx->mlp;
  std::vector<int> perm, tt, ro;
  int off[5];
  mlp_tiles_host(ctx->h_types, perm, tt, ro, off);
  M.tiles.rows = (int)perm.size();
  M.tiles.ntile = (int)tt.size();
  CK(cudaMemcpyAsync(M.tiles.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.tiles.tile_type, tt.data(), tt.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.tiles.rows_off, ro.data(), ro.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.types, ctx->h_types.data(), ctx->n * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.off, off, sizeof(off), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return REAXFF_OK;
}

int mlp_alloc(reaxff_ctx* ctx) {
  auto& M = ctx->mlp;
  if (M.alloc) return REAXFF_OK;
  const int n = ctx->n;
  for (int t : ctx->h_types)
    if (t < 0 || t >= rx::MLP_NT) return fail(ctx, REAXFF_E_INVALID, "the learned warm start needs element types 0..3");
  DevBuf& B = M.buf;
  const size_t NPT = (size_t)rx::MLP_NT * rx::MLP_NPAR;
  M.theta = B.alloc<float>(NPT); M.madam = B.alloc<float>(NPT); M.vadam = B.alloc<float>(NPT); M.grad = B.alloc<float>(NPT);
  M.mean = B.alloc<float>(rx::MLP_NF); M.inv = B.alloc<float>(rx::MLP_NF);
  M.loss = B.alloc<double>(1);
  M.D = B.alloc<float>((size_t)n * rx::MLP_NF);
  M.y = B.alloc<float>(n);
  M.types = B.alloc<int>(n);
  M.off = B.alloc<int>(rx::MLP_NT + 1);
  std::vector<int> perm, tt, ro;
  int off[5];
  mlp_tiles_host(ctx->h_types, perm, tt, ro, off);
  M.tiles.rows = (int)perm.size();
  M.tiles.ntile = (int)tt.size();
  M.tiles.perm = B.alloc<int>(perm.size());
  M.tiles.tile_type = B.alloc<int>(ctx->n / 128 + rx::MLP_NT + 1);   // tiles: at most n/128 + one per element
  M.tiles.rows_off = B.alloc<int>(ctx->n / 128 + rx::MLP_NT + 2);
  M.inf.Xp = B.alloc_bytes((size_t)n * rx::MLP_NF * 2);
  M.inf.W1t = B.alloc_bytes((size_t)rx::MLP_NT * rx::MLP_HID * rx::MLP_NF * 2);
  M.inf.W2t = B.alloc_bytes((size_t)rx::MLP_NT * rx::MLP_HID * rx::MLP_HID * 2);
  M.inf.fp = B.alloc<float>((size_t)rx::MLP_NT * (3 * rx::MLP_HID + 1));
  float** sc[] = {&M.scr.z1, &M.scr.z2, &M.scr.dz1, &M.scr.dz2};
  for (float** p : sc) *p = B.alloc<float>((size_t)n * rx::MLP_HID);
  M.scr.y = B.alloc<float>(n);
  M.scr.l = B.alloc<float>(n);
  M.scr.part = B.alloc<float>((size_t)((n + rx::MLP_WG_CHUNK - 1) / rx::MLP_WG_CHUNK) * rx::MLP_NT * rx::MLP_NPAR);
  if (B.err != cudaSuccess) {
    B.free_all();
    return fail(ctx, REAXFF_E_CUDA, "learned warm start allocation: " + cuda_err_str(B.err));
  }
  int rc = mlp_tiles_upload(ctx);
  if (rc) return rc;
  CK(cudaMemsetAsync(M.theta, 0, NPT * sizeof(float), ctx->st));
  CK(cudaMemsetAsync(M.madam, 0, NPT * sizeof(float), ctx->st));
  CK(cudaMemsetAsync(M.vadam, 0, NPT * sizeof(float), ctx->st));
  CK(cudaMemsetAsync(M.mean, 0, rx::MLP_NF * sizeof(float), ctx->st));
  CK(cudaMemsetAsync(M.inv, 0, rx::MLP_NF * sizeof(float), ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (rx::mlp_tc_setup() != 0) return fail(ctx, REAXFF_E_CUDA, "tensor-core kernel shared-memory attribute");
  M.alloc = true;
  return REAXFF_OK;
}

// descriptors of the current positions (lists built or reused as the forces left them)
int mlp_current_descriptors(reaxff_ctx* ctx) {
  if (!ctx->lists_valid) {
    int rc = build_lists_impl(ctx);
    if (rc) return rc;
  }
  rx::mlp_descriptors(launch_of(ctx), ctx->sys, ctx->far, ctx->mlp.D);
  return REAXFF_OK;
}

// temporary device copies of caller data for the test entry points
struct Tmp {
  std::vector<void*> p;
  ~Tmp() { for (void* q : p) cudaFree(q); }
  template <typename T> T* up(reaxff_ctx* ctx, const T* host, size_t count) {
    void* d = nullptr;
    if (cudaMalloc(&d, (count ? count : 1) * sizeof(T)) != cudaSuccess) return nullptr;
    p.push_back(d);
    if (host && cudaMemcpyAsync(d, host, count * sizeof(T), cudaMemcpyHostToDevice, ctx->st) != cudaSuccess) return nullptr;
    return (T*)d;
  }
};

__global__ void k_q_to_float(const double* q, float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)q[i];
}
}  // namespace

extern "C" {

int reaxff_mlp_init(reaxff_ctx* ctx, uint64_t seed) {
  if (!ctx) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  auto& M = ctx->mlp;
  std::vector<float> th((size_t)rx::MLP_NT * rx::MLP_NPAR, 0.0f);
  uint64_t st = seed;
  const int NF = rx::MLP_NF, H = rx::MLP_HID;
  for (int t = 0; t < rx::MLP_NT; ++t) {
    float* w = th.data() + (size_t)t * rx::MLP_NPAR;
    auto normal = [&]() {                                 // Box-Muller, draws in a fixed order
      const double u1 = u01(st), u2 = u01(st);
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int k = 0; k < NF * H; ++k) w[k] = (float)(normal() * std::sqrt(1.0 / NF));
    for (int k = 0; k < H * H; ++k) w[NF * H + H + k] = (float)(normal() * std::sqrt(1.0 / H));
    for (int k = 0; k < H; ++k) w[NF * H + H + H * H + H + k] = (float)(normal() * std::sqrt(1.0 / H));
  }
  CK(cudaMemcpyAsync(M.theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(M.madam, 0, th.size() * sizeof(float), ctx->st));
  CK(cudaMemsetAsync(M.vadam, 0, th.size() * sizeof(float), ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  M.adam_step = 0;
  M.fresh = true;
  M.ready = false;
  return REAXFF_OK;
}

int reaxff_mlp_set_params(reaxff_ctx* ctx, const float* theta, const float* mean, const float* inv_std) {
  if (!ctx || !theta || !mean || !inv_std) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  auto& M = ctx->mlp;
  CK(cudaMemcpyAsync(M.theta, theta, (size_t)rx::MLP_NT * rx::MLP_NPAR * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.mean, mean, rx::MLP_NF * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(M.inv, inv_std, rx::MLP_NF * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
  rx::mlp_weights(launch_of(ctx), M.theta, M.inf);
  CK(cudaStreamSynchronize(ctx->st));
  M.ready = true;
  M.fresh = false;
  drop_graph(ctx);
  return REAXFF_OK;
}

int reaxff_mlp_get_params(reaxff_ctx* ctx, float* theta, float* mean, float* inv_std) {
  if (!ctx) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  auto& M = ctx->mlp;
  if (theta) CK(cudaMemcpyAsync(theta, M.theta, (size_t)rx::MLP_NT * rx::MLP_NPAR * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  if (mean) CK(cudaMemcpyAsync(mean, M.mean, rx::MLP_NF * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  if (inv_std) CK(cudaMemcpyAsync(inv_std, M.inv, rx::MLP_NF * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return REAXFF_OK;
}

int reaxff_mlp_descriptors(reaxff_ctx* ctx, float* D) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
  if ((rc = mlp_current_descriptors(ctx))) return rc;
  int flags = 0;
  if ((rc = read_err(ctx, &flags))) return rc;
  if (flags & ERR_CAP_DESC) return fail(ctx, REAXFF_E_CAPACITY, "more neighbours than the descriptor kernel keeps");
  if (D) {
    std::vector<float> Ds(ctx->perm.empty() ? 0 : (size_t)ctx->n * rx::MLP_NF);
    CK(cudaMemcpyAsync(Ds.empty() ? D : Ds.data(), ctx->mlp.D, (size_t)ctx->n * rx::MLP_NF * sizeof(float),
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (!Ds.empty()) rows_to_caller(ctx, Ds.data(), D, rx::MLP_NF);
  }
  return REAXFF_OK;
}

int reaxff_mlp_infer(reaxff_ctx* ctx, const float* D, const int32_t* types, int64_t m, float* y) {
  if (!ctx || !D || !types || !y || m <= 0 || m > (1 << 30)) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  std::vector<int> ty(types, types + m), perm, tt, ro;
  for (int t : ty)
    if (t < 0 || t >= rx::MLP_NT) return fail(ctx, REAXFF_E_INVALID, "element types must be 0..3");
  int off[5];
  mlp_tiles_host(ty, perm, tt, ro, off);
  Tmp T;
  float* Dd = T.up(ctx, D, (size_t)m * rx::MLP_NF);
  float* yd = T.up<float>(ctx, nullptr, m);
  rx::MlpTiles tl{(int)perm.size(), (int)tt.size(), T.up(ctx, perm.data(), perm.size()), T.up(ctx, tt.data(), tt.size()),
                  T.up(ctx, ro.data(), ro.size())};
  rx::MlpInfer inf = ctx->mlp.inf;
  inf.Xp = T.up<char>(ctx, nullptr, (size_t)m * rx::MLP_NF * 2);
  if (!Dd || !yd || !tl.perm || !tl.tile_type || !tl.rows_off || !inf.Xp) return fail(ctx, REAXFF_E_CUDA, "allocation");
  CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
  rx::mlp_weights(launch_of(ctx), ctx->mlp.theta, inf);
  rx::mlp_infer(launch_of(ctx), Dd, tl, ctx->mlp.mean, ctx->mlp.inv, inf, yd, ctx->sys.err, ctx->nsm);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(y, yd, m * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  int flags = 0;
  if ((rc = read_err(ctx, &flags))) return rc;
  if (flags & ERR_TIMEOUT) return fail(ctx, REAXFF_E_TIMEOUT, "tensor-core wait hit its spin limit");
  return REAXFF_OK;
}

int reaxff_mlp_loss_grad(reaxff_ctx* ctx, const float* D, const int32_t* types, const float* q, int64_t m, float* grad,
                         double* loss) {
  if (!ctx || !D || !types || !q || m <= 0 || m > (1 << 30)) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  std::vector<int> ty(types, types + m), perm, tt, ro;
  for (int t : ty)
    if (t < 0 || t >= rx::MLP_NT) return fail(ctx, REAXFF_E_INVALID, "element types must be 0..3");
  int off[5];
  mlp_tiles_host(ty, perm, tt, ro, off);
  Tmp T;
  float* Dd = T.up(ctx, D, (size_t)m * rx::MLP_NF);
  float* qd = T.up(ctx, q, m);
  int* td = T.up(ctx, ty.data(), m);
  int* pd = T.up(ctx, perm.data(), perm.size());
  int* od = T.up(ctx, off, 5);
  rx::MlpScratch w{};
  float** sc[] = {&w.z1, &w.z2, &w.dz1, &w.dz2};
  for (float** p : sc) *p = T.up<float>(ctx, nullptr, (size_t)m * rx::MLP_HID);
  w.y = T.up<float>(ctx, nullptr, m);
  w.l = T.up<float>(ctx, nullptr, m);
  w.part = T.up<float>(ctx, nullptr, (size_t)((m + rx::MLP_WG_CHUNK - 1) / rx::MLP_WG_CHUNK) * rx::MLP_NT * rx::MLP_NPAR);
  if (!Dd || !qd || !td || !pd || !od || !w.z1 || !w.z2 || !w.dz1 || !w.dz2 || !w.y || !w.l || !w.part)
    return fail(ctx, REAXFF_E_CUDA, "allocation");
  auto& M = ctx->mlp;
  rx::mlp_loss_grad(launch_of(ctx), Dd, td, pd, od, qd, (int)m, M.theta, M.mean, M.inv, w, M.grad, M.loss);
  CK(cudaGetLastError());
  if (grad) CK(cudaMemcpyAsync(grad, M.grad, (size_t)rx::MLP_NT * rx::MLP_NPAR * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  double l = 0.0;
  CK(cudaMemcpyAsync(&l, M.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (loss) *loss = l;
  return REAXFF_OK;
}

int reaxff_mlp_adam_step(reaxff_ctx* ctx, const float* grad, double lr) {
  if (!ctx || !grad || !(lr > 0)) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  auto& M = ctx->mlp;
  CK(cudaMemcpyAsync(M.grad, grad, (size_t)rx::MLP_NT * rx::MLP_NPAR * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
  rx::mlp_adam(launch_of(ctx), M.theta, M.grad, M.madam, M.vadam, ++M.adam_step, (float)lr);
  rx::mlp_weights(launch_of(ctx), M.theta, M.inf);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->st));
  return REAXFF_OK;
}

int reaxff_mlp_reserve(reaxff_ctx* ctx, int32_t nsnap) {
  if (!ctx || nsnap < 1) return REAXFF_E_INVALID;
  int rc = mlp_alloc(ctx);
  if (rc) return rc;
  auto& M = ctx->mlp;
  M.data.free_all();
  M.TD = M.data.alloc<float>((size_t)nsnap * ctx->n * rx::MLP_NF);
  M.TQ = M.data.alloc<float>((size_t)nsnap * ctx->n);
  if (M.data.err != cudaSuccess) {
    M.data.free_all();
    M.cap = M.count = 0;
    return fail(ctx, REAXFF_E_CUDA, "training-set allocation: " + cuda_err_str(M.data.err));
  }
  M.cap = nsnap;
  M.count = 0;
  return REAXFF_OK;
}

int reaxff_mlp_collect(reaxff_ctx* ctx) {
  if (!ctx) return REAXFF_E_INVALID;
  auto& M = ctx->mlp;
  if (!M.alloc || M.count >= M.cap) return fail(ctx, REAXFF_E_CAPACITY, "training set full (reaxff_mlp_reserve)");
  int rc;
  if (!ctx->forces_valid) {
    if ((rc = forces_impl(ctx, true))) return rc;
  }
  CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
  if ((rc = mlp_current_descriptors(ctx))) return rc;
  const size_t n = ctx->n;
  CK(cudaMemcpyAsync(M.TD + (size_t)M.count * n * rx::MLP_NF, M.D, n * rx::MLP_NF * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
  k_q_to_float<<<(ctx->n + 255) / 256, 256, 0, ctx->st>>>(ctx->sys.q, M.TQ + (size_t)M.count * n, ctx->n);
  CK(cudaGetLastError());
  int flags = 0;
  if ((rc = read_err(ctx, &flags))) return rc;
  if (flags & ERR_CAP_DESC) return fail(ctx, REAXFF_E_CAPACITY, "more neighbours than the descriptor kernel keeps");
  ++M.count;
  return REAXFF_OK;
}

int reaxff_mlp_train(reaxff_ctx* ctx, int32_t epochs, double lr, double* loss_out) {
  if (!ctx || epochs < 1 || !(lr > 0)) return REAXFF_E_INVALID;
  auto& M = ctx->mlp;
  if (!M.alloc || M.count < 1) return fail(ctx, REAXFF_E_STATE, "no training snapshots (reaxff_mlp_collect)");
  rx::Launch L = launch_of(ctx);
  const size_t n = ctx->n;
  rx::mlp_stats(L, M.TD, (int64_t)M.count * n, M.mean, M.inv);
  if (M.fresh) {
    // output bias of each element's network = its mean training charge
    std::vector<float> q((size_t)M.count * n);
    CK(cudaMemcpyAsync(q.data(), M.TQ, q.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int t = 0; t < rx::MLP_NT; ++t) {
      double sum = 0.0;
      size_t c = 0;
      for (size_t k = 0; k < q.size(); ++k)
        if (ctx->h_types[k % n] == t) { sum += q[k]; ++c; }
      const float b3 = c ? (float)(sum / c) : 0.0f;
      CK(cudaMemcpyAsync(M.theta + (size_t)t * rx::MLP_NPAR + rx::MLP_NPAR - 1, &b3, sizeof(float), cudaMemcpyHostToDevice, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    M.fresh = false;
  }
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    double sum = 0.0;
    for (int sidx = 0; sidx < M.count; ++sidx) {
      rx::mlp_loss_grad(L, M.TD + (size_t)sidx * n * rx::MLP_NF, M.types, M.tiles.perm, M.off, M.TQ + (size_t)sidx * n,
                        ctx->n, M.theta, M.mean, M.inv, M.scr, M.grad, M.loss);
      rx::mlp_adam(L, M.theta, M.grad, M.madam, M.vadam, ++M.adam_step, (float)lr);
      if (ep == epochs - 1) {
        double l = 0.0;
        CK(cudaMemcpyAsync(&l, M.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        sum += l;
      }
    }
    last = sum / M.count;
  }
  rx::mlp_weights(L, M.theta, M.inf);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->st));
  M.ready = true;
  drop_graph(ctx);                        // the step graph now runs the network
  if (loss_out) *loss_out = last;
  return REAXFF_OK;
}

int reaxff_mlp_predict(reaxff_ctx* ctx, double* q) {
  if (!ctx || !q) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  auto& M = ctx->mlp;
  if (!M.alloc || !M.ready) return fail(ctx, REAXFF_E_STATE, "the network has no parameters (train or set them)");
  int rc;
  CK(cudaMemsetAsync(ctx->sys.err, 0, sizeof(int), ctx->st));
  if ((rc = mlp_current_descriptors(ctx))) return rc;
  rx::mlp_infer(launch_of(ctx), M.D, M.tiles, M.mean, M.inv, M.inf, M.y, ctx->sys.err, ctx->nsm);
  CK(cudaGetLastError());
  std::vector<float> y(ctx->n);
  CK(cudaMemcpyAsync(y.data(), M.y, ctx->n * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  int flags = 0;
  if ((rc = read_err(ctx, &flags))) return rc;
  if (flags & ERR_TIMEOUT) return fail(ctx, REAXFF_E_TIMEOUT, "tensor-core wait hit its spin limit");
  if (flags & ERR_CAP_DESC) return fail(ctx, REAXFF_E_CAPACITY, "more neighbours than the descriptor kernel keeps");
  for (int i = 0; i < ctx->n; ++i) q[ext_of(ctx, i)] = y[i];
  return REAXFF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ species analysis
namespace {
// species analysis over a bond view (bonds with bo > threshold); bo_double: the view's bo
// array is double, else the path type
int species_impl(reaxff_ctx* ctx, const BondList& bl, bool bo_double, const double* bo_threshold,
                 int32_t* mol_id, int64_t* nmol, int32_t cap, int32_t* species, int32_t* nspecies) {
  const int n = ctx->n;
  rx::SpeciesBuf& b = ctx->sp;
  if (!b.lab) {
    DevBuf& B = ctx->spbuf;
    b.lab = B.alloc<int>(n); b.rank = B.alloc<int>(n); b.mol = B.alloc<int>(n);
    b.cnt = B.alloc<int>((size_t)n * MAXT); b.mrep = B.alloc<int>(n);
    b.boff = B.alloc<int>(n / 1024 + 2); b.nmol = B.alloc<int>(1); b.changed = B.alloc<int>(1);
    ctx->sp_thr = B.alloc<double>(MAXT * MAXT);
    if (B.err != cudaSuccess || cudaMallocHost(&b.h_changed, sizeof(int)) != cudaSuccess) {
      B.free_all();
      b = rx::SpeciesBuf{};
      return fail(ctx, REAXFF_E_CUDA, "species buffers");
    }
  }
  double thr[MAXT * MAXT];
  for (int k = 0; k < MAXT * MAXT; ++k) thr[k] = bo_threshold ? bo_threshold[k] : 0.3;
  CK(cudaMemcpyAsync(ctx->sp_thr, thr, sizeof(thr), cudaMemcpyHostToDevice, ctx->st));
  rx::Launch L = launch_of(ctx);
  const int passes = bo_double ? rx::species_components<double>(L, ctx->sys, bl, ctx->sp_thr, b, 256)
                               : rx::species_components<float>(L, ctx->sys, bl, ctx->sp_thr, b, 256);
  CK(cudaGetLastError());
  if (passes < 0) return fail(ctx, REAXFF_E_NOT_CONVERGED, "species components did not settle in 256 passes");
  rx::species_molecules(L, ctx->sys, b);
  CK(cudaGetLastError());
  int M = 0;
  CK(cudaMemcpyAsync(&M, b.nmol, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  std::vector<int> cnt((size_t)M * MAXT), mrep(M);
  CK(cudaMemcpyAsync(cnt.data(), b.cnt, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(mrep.data(), b.mrep, mrep.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  std::vector<int> ms(mol_id && !ctx->perm.empty() ? n : 0);
  if (mol_id) CK(cudaMemcpyAsync(ms.empty() ? mol_id : ms.data(), b.mol, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (!ms.empty()) {
    // stored in cell order: number the molecules by their smallest index in the caller's order
    std::vector<int> first(M, n), order(M), id(M);
    for (int k = 0; k < n; ++k) first[ms[k]] = std::min(first[ms[k]], ext_of(ctx, k));
    for (int m = 0; m < M; ++m) order[m] = m;
    std::sort(order.begin(), order.end(), [&](int u, int v) { return first[u] < first[v]; });
    for (int m = 0; m < M; ++m) id[order[m]] = m;
    for (int k = 0; k < n; ++k) mol_id[ext_of(ctx, k)] = id[ms[k]];
  }
  // the summary: molecules per (replica, element counts), in that order
  constexpr int W = MAXT + 2;
  std::vector<std::array<int, MAXT + 1>> keys(M);
  for (int m = 0; m < M; ++m) {
    keys[m][0] = mrep[m];
    for (int t = 0; t < MAXT; ++t) keys[m][1 + t] = cnt[(size_t)m * MAXT + t];
  }
  std::sort(keys.begin(), keys.end());
  int ns = 0;
  for (int m = 0; m < M;) {
    int e = m;
    while (e < M && keys[e] == keys[m]) ++e;
    if (ns < cap) {
      for (int q = 0; q <= MAXT; ++q) species[ns * W + q] = keys[m][q];
      species[ns * W + MAXT + 1] = e - m;
    }
    ++ns;
    m = e;
  }
  if (nmol) *nmol = M;
  if (nspecies) *nspecies = ns;
  if (ns > cap) return fail(ctx, REAXFF_E_CAPACITY, "more species than cap (count in *nspecies)");
  return REAXFF_OK;
}

// the averages of the samples so far into avg.avg (needs at least one sample)
int bo_average_ready(reaxff_ctx* ctx) {
  if (ctx->avg_samples == 0) return fail(ctx, REAXFF_E_STATE, "no bond-order samples");
  int over = 0;
  CK(cudaMemcpyAsync(&over, ctx->avg.over, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (over) return fail(ctx, REAXFF_E_CAPACITY, "an atom met more distinct bonded pairs than the average table holds");
  rx::Launch L = launch_of(ctx);
  rx::bo_average_finish(L, ctx->n, ctx->avg, 1.0 / (double)ctx->avg_samples);
  CK(cudaGetLastError());
  return REAXFF_OK;
}
}  // namespace

extern "C" {

int reaxff_species(reaxff_ctx* ctx, const double* bo_threshold, int32_t* mol_id, int64_t* nmol, int32_t cap,
                   int32_t* species, int32_t* nspecies) {
  if (!ctx || cap < 0 || (cap > 0 && !species)) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  int rc;
  if (!ctx->forces_valid) {
    if ((rc = forces_impl(ctx, true))) return rc;
  }
  return species_impl(ctx, ctx->bond, ctx->fp64, bo_threshold, mol_id, nmol, cap, species, nspecies);
}

int reaxff_bo_average_reset(reaxff_ctx* ctx) {
  if (!ctx) return REAXFF_E_INVALID;
  ctx->avg_samples = 0;
  if (ctx->avg.cnt) {
    CK(cudaMemsetAsync(ctx->avg.cnt, 0, ctx->n * sizeof(int), ctx->st));
    CK(cudaMemsetAsync(ctx->avg.over, 0, sizeof(int), ctx->st));
  }
  return REAXFF_OK;
}

int reaxff_bo_average_sample(reaxff_ctx* ctx) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  int rc;
  if (!ctx->forces_valid) {
    if ((rc = forces_impl(ctx, true))) return rc;
  }
  rx::BoAvg& A = ctx->avg;
  if (!A.cnt) {
    DevBuf& B = ctx->avgbuf;
    const int n = ctx->n;
    A.cap = std::max(48, 2 * ctx->cap_bond);
    A.cnt = B.alloc<int>(n);
    A.j = B.alloc<int>((size_t)n * A.cap);
    A.s = B.alloc<uint8_t>((size_t)n * A.cap);
    A.sum = B.alloc<double>((size_t)n * A.cap);
    A.avg = B.alloc<double>((size_t)n * A.cap);
    A.over = B.alloc<int>(1);
    if (B.err != cudaSuccess) {
      B.free_all();
      A = rx::BoAvg{};
      return fail(ctx, REAXFF_E_CUDA, "bond-order average buffers");
    }
    ctx->avg_samples = 0;
    CK(cudaMemsetAsync(A.cnt, 0, n * sizeof(int), ctx->st));
    CK(cudaMemsetAsync(A.over, 0, sizeof(int), ctx->st));
  }
  rx::Launch L = launch_of(ctx);
  if (ctx->fp64) rx::bo_average_sample<double>(L, ctx->sys, ctx->bond, A);
  else rx::bo_average_sample<float>(L, ctx->sys, ctx->bond, A);
  CK(cudaGetLastError());
  ++ctx->avg_samples;
  return REAXFF_OK;
}

int64_t reaxff_bo_average_samples(reaxff_ctx* ctx) { return ctx ? ctx->avg_samples : -1; }

int reaxff_get_bo_average(reaxff_ctx* ctx, int64_t capacity, int64_t* count, int32_t* i_out, int32_t* j_out,
                          int8_t* shift, double* avg_out) {
  if (!ctx || !count) return REAXFF_E_INVALID;
  int rc = bo_average_ready(ctx);
  if (rc) return rc;
  const int n = ctx->n;
  const rx::BoAvg& A = ctx->avg;
  std::vector<int> cnt(n);
  CK(cudaMemcpyAsync(cnt.data(), A.cnt, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  int64_t tot = 0;
  for (int i = 0; i < n; ++i) tot += cnt[i];
  *count = tot;
  if (capacity == 0 && !i_out) return REAXFF_OK;
  if (capacity < tot || !i_out || !j_out || !shift || !avg_out)
    return fail(ctx, REAXFF_E_INVALID, "output capacity too small");
  std::vector<int> jj((size_t)n * A.cap);
  std::vector<uint8_t> ss((size_t)n * A.cap);
  std::vector<double> av((size_t)n * A.cap);
  CK(cudaMemcpyAsync(jj.data(), A.j, jj.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(ss.data(), A.s, ss.size(), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(av.data(), A.avg, av.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  int64_t k = 0;
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < cnt[i]; ++m, ++k) {
      const size_t e = (size_t)i * A.cap + m;
      i_out[k] = ext_of(ctx, i);
      j_out[k] = ext_of(ctx, jj[e]);
      const int c = ss[e];
      shift[3 * k + 0] = (int8_t)(c / 9 - 1);
      shift[3 * k + 1] = (int8_t)((c / 3) % 3 - 1);
      shift[3 * k + 2] = (int8_t)(c % 3 - 1);
      avg_out[k] = av[e];
    }
  return REAXFF_OK;
}

int reaxff_species_average(reaxff_ctx* ctx, const double* bo_threshold, int32_t* mol_id, int64_t* nmol,
                           int32_t cap, int32_t* species, int32_t* nspecies) {
  if (!ctx || cap < 0 || (cap > 0 && !species)) return REAXFF_E_INVALID;
  int rc = bo_average_ready(ctx);
  if (rc) return rc;
  BondList v{};
  v.cap = ctx->avg.cap;
  v.cnt = ctx->avg.cnt;
  v.j = ctx->avg.j;
  v.s = ctx->avg.s;
  v.bo = ctx->avg.avg;
  return species_impl(ctx, v, true, bo_threshold, mol_id, nmol, cap, species, nspecies);
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace {
template <typename R> const DParams<R>* params_ptr(reaxff_ctx* ctx);
template <> const DParams<double>* params_ptr<double>(reaxff_ctx* ctx) { return ctx->Pd; }
template <> const DParams<float>* params_ptr<float>(reaxff_ctx* ctx) { return ctx->Pf; }

// mean device time (ms) of `launch` over `runs` runs after `warm` warm-up runs; +inf if it
// fails
template <typename F> float time_launch(reaxff_ctx* ctx, F&& launch, int warm = 2, int runs = 8) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 1e30f;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 1e30f; }
  for (int k = 0; k < warm; ++k) launch();
  cudaEventRecord(a, ctx->st);
  for (int k = 0; k < runs; ++k) launch();
  cudaEventRecord(b, ctx->st);
  float ms = 1e30f;
  if (cudaEventSynchronize(b) == cudaSuccess && cudaGetLastError() == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  else ms = 1e30f;
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / (float)runs;
}

// Where the QEq solve runs (schedule entry 7), timed on MD steps through the captured step
// graph: whole force evaluations rank the close candidates (512 threads on every SM, or
// 1024-thread blocks on part of the SMs) differently from the steps they are for. Every
// candidate starts from the same state (positions, velocities, solution history: the
// rollback snapshot, kept aside), runs 3 warm-up steps of 0.1 fs and three timed windows of
// 16, and the state is restored after it; each candidate's fastest window counts. Windows
// this early in a trajectory still rank placements within a few per cent of each other
// unlike the steady state (petn32k: half of the SMs 1.6 % faster over steps 4-51, 3.5 %
// slower over steps 148-547, both reproducible to 0.1 %), so the 512-thread placement
// beside the terms (1) is kept unless another is more than 3 % faster.
void tune_solve_placement(reaxff_ctx* ctx) {
  rx::Tune& T = ctx->tune;
  rx::Launch L = launch_of(ctx);
  const size_t nd = (6 + 2 * (size_t)rx::QEQ_HIST) * ctx->n;
  double* keep = nullptr;
  int* keep_i = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&keep, nd * sizeof(double)) != cudaSuccess || cudaMalloc(&keep_i, 4 * sizeof(int)) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (keep) cudaFree(keep);
    if (keep_i) cudaFree(keep_i);
    if (a) cudaEventDestroy(a);
    return;                                               // keeps the default placement
  }
  const bool had_forces = ctx->forces_valid;
  rx::snapshot(L, ctx->sys, ctx->Q.hist_s, 2 * rx::QEQ_HIST * ctx->n, ctx->Q.hst, ctx->snap, ctx->snap_i, 0);
  cudaMemcpyAsync(keep, ctx->snap, nd * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st);
  cudaMemcpyAsync(keep_i, ctx->snap_i, 4 * sizeof(int), cudaMemcpyDeviceToDevice, ctx->st);
  auto restore = [&] {
    cudaMemcpyAsync(ctx->snap, keep, nd * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st);
    cudaMemcpyAsync(ctx->snap_i, keep_i, 4 * sizeof(int), cudaMemcpyDeviceToDevice, ctx->st);
    rx::snapshot(L, ctx->sys, ctx->Q.hist_s, 2 * rx::QEQ_HIST * ctx->n, ctx->Q.hst, ctx->snap, ctx->snap_i, 1);
    cudaMemsetAsync(ctx->sys.img, 0, 3 * (size_t)ctx->n * sizeof(int), ctx->st);
    cudaMemsetAsync(ctx->sys.rebuild, 1, sizeof(int), ctx->st);
    ctx->forces_valid = false;
    ctx->lists_valid = false;
  };
  float ms_of[rx::QEQ_PLACEMENTS];
  for (int c = 0; c < rx::QEQ_PLACEMENTS; ++c) {
    T.qeq_overlap = c;
    drop_graph(ctx);
    float ms = 1e30f;
    int flags = 0;
    if (forces_impl(ctx, true) == REAXFF_OK && run_unchecked(ctx, 3, 0.1, nullptr, &flags) == REAXFF_OK && !flags) {
      for (int w = 0; w < 3; ++w) {
        cudaEventRecord(a, ctx->st);
        const int rc = run_unchecked(ctx, 16, 0.1, nullptr, &flags);
        cudaEventRecord(b, ctx->st);
        float t = 1e30f;
        if (rc != REAXFF_OK || flags || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
          ms = 1e30f;
          break;
        }
        ms = std::min(ms, t / 16.0f);
      }
    }
    cudaGetLastError();
    restore();
    ms_of[c] = ms;
  }
  int arg = 1;
  for (int c = 0; c < rx::QEQ_PLACEMENTS; ++c)
    if (ms_of[c] < ms_of[arg] && (arg != 1 || ms_of[c] < 0.97f * ms_of[1])) arg = c;
  T.qeq_overlap = arg;
  drop_graph(ctx);
  cudaStreamSynchronize(ctx->st);
  cudaFree(keep);
  cudaFree(keep_i);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (had_forces && forces_impl(ctx, true) != REAXFF_OK) cudaGetLastError();
}

template <typename R> void tune_all(reaxff_ctx* ctx) {
  rx::Launch L = launch_of(ctx);
  const DParams<R>* P = params_ptr<R>(ctx);
  rx::Tune& T = ctx->tune;
  auto pick = [&](int& knob, std::initializer_list<int> cands, auto&& run) {
    float best = 1e30f;
    int arg = knob;
    for (int c : cands) {
      knob = c;
      const float ms = time_launch(ctx, run);
      if (ms < best) { best = ms; arg = c; }
    }
    knob = arg;
  };
  pick(T.tors_lanes, {2, 4, 8}, [&] { rx::torsions<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); });
  pick(T.nb_block, {128, 256, 512}, [&] { rx::nonbonded<R>(L, ctx->sys, ctx->far, ctx->acc, P, ctx->mask); });
  if (!ctx->fp64)
    pick(T.ang_lanes, {8, 16, 32}, [&] { rx::angles<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); });
  pick(T.ang_block, {64, 128, 256}, [&] { rx::angles<R>(L, ctx->sys, ctx->bond, ctx->aq, ctx->acc, P, ctx->mask); });
  pick(T.hb_block, {64, 128, 256}, [&] { rx::hbonds<R>(L, ctx->sys, ctx->bond, ctx->hb, ctx->acc, P, ctx->mask); });
  if (ctx->use_skin)
    pick(T.cf_block, {128, 256, 512}, [&] {
      rx::cand_filter<R>(L, ctx->sys, ctx->cand, ctx->far, ctx->hb, P, ctx->far_margin, ctx->near_margin, ctx->hb_margin);
    });
  pick(T.bl_block, {128, 256, 512}, [&] {
    cudaMemsetAsync(ctx->bond.ncanon, 0, sizeof(int), ctx->st);
    rx::bond_list<R>(L, ctx->sys, ctx->far, ctx->bond, ctx->hb, ctx->aq, P, ctx->Pd, ctx->use_skin);
  });
  // the solve beside the charge-free terms or before them: whole force evaluations timed.
  // Repeated at the same positions, a warm-started solve would converge at once; each timed
  // solve instead starts without history and is capped at 8 SpMVs, about those of an MD step
  // (the capped solves' flags are cleared by the checked evaluation that follows tuning)
  if (!ctx->fp64) {
    tune_solve_placement(ctx);
    const int mi = ctx->ho.qeq_max_iter;
    ctx->ho.qeq_max_iter = 7;
    auto whole = [&] {
      cudaMemsetAsync(ctx->Q.hst + 2, 0, sizeof(int), ctx->st);
      forces_impl(ctx, true, true, false);
    };
    if (T.qeq_overlap != 0) {
      // beside the resident solve the charge-free kernels get fewer registers and warps per
      // SM than when timed alone above: their launch shapes are picked again by whole
      // overlapped force evaluations
      // the candidates of each entry interleaved over 4 rounds (a warm-up and 3 timed
      // evaluations each) and each candidate's fastest round counted, so that a drift of
      // the GPU's state during the pass favours no candidate by its place in the order
      auto pick_rounds = [&](int& knob, std::initializer_list<int> cands) {
        const std::vector<int> cs(cands);
        std::vector<float> best(cs.size(), 1e30f);
        for (int round = 0; round < 4; ++round)
          for (size_t c = 0; c < cs.size(); ++c) {
            knob = cs[c];
            best[c] = std::min(best[c], time_launch(ctx, whole, 1, 3));
          }
        size_t arg = 0;
        for (size_t c = 1; c < cs.size(); ++c)
          if (best[c] < best[arg]) arg = c;
        knob = cs[arg];
      };
      pick_rounds(T.tors_lanes, {1, 2, 4, 8});
      pick_rounds(T.ang_lanes, {4, 8, 16, 32});
      pick_rounds(T.ang_block, {64, 128, 256});
      pick_rounds(T.hb_block, {64, 128, 256});
      pick_rounds(T.nb_block, {128, 256, 512});
      pick_rounds(T.bl_block, {128, 256, 512});
    }
    ctx->ho.qeq_max_iter = mi;
    cudaMemsetAsync(ctx->Q.hst + 2, 0, sizeof(int), ctx->st);
  }
}

// a schedule read from a cache file: every entry one the tuner can pick (a line edited by hand
// or from another version is ignored, and the context is tuned again)
bool tune_valid(const rx::Tune& t) {
  auto in = [](int v, std::initializer_list<int> set) {
    for (int c : set)
      if (v == c) return true;
    return false;
  };
  return in(t.tors_lanes, {1, 2, 4, 8}) && in(t.ang_lanes, {4, 8, 16, 32}) && in(t.nb_block, {128, 256, 512}) &&
         in(t.cf_block, {128, 256, 512}) && in(t.bl_block, {128, 256, 512}) && in(t.ang_block, {64, 128, 256}) &&
         in(t.hb_block, {64, 128, 256}) && t.qeq_overlap >= 0 && t.qeq_overlap < rx::QEQ_PLACEMENTS;
}

std::string tune_key(reaxff_ctx* ctx) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp pr{};
  cudaGetDeviceProperties(&pr, dev);
  char buf[256];
  snprintf(buf, sizeof(buf), "n=%d nrep=%d prec=%d skin=%d sm=%d.%d sms=%d", ctx->n, ctx->nrep, ctx->fp64 ? 0 : 1,
           ctx->use_skin ? 1 : 0, pr.major, pr.minor, pr.multiProcessorCount);
  return buf;
}
}  // namespace

extern "C" {

int reaxff_extrap_weights(int32_t predictor, double* w) {
  if (!w || predictor < 0 || predictor >= rx::QEQ_NPRED) return REAXFF_E_INVALID;
  std::vector<double> v;
  extrap_weights(predictor, v);
  std::copy(v.begin(), v.end(), w);
  return REAXFF_OK;
}

int reaxff_autotune(reaxff_ctx* ctx, const char* cache_path, int32_t* schedule) {
  if (!ctx) return REAXFF_E_INVALID;
  if (!ctx->have_pos) return fail(ctx, REAXFF_E_STATE, "positions not set");
  const std::string key = tune_key(ctx);
  bool found = false;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        rx::Tune t{};
        char k[256];
        if (sscanf(line, "reaxff-tune %255[^|]| tors=%d nb=%d cf=%d bl=%d ang=%d hb=%d angl=%d qov=%d", k,
                   &t.tors_lanes, &t.nb_block, &t.cf_block, &t.bl_block, &t.ang_block, &t.hb_block, &t.ang_lanes,
                   &t.qeq_overlap) == 9 && tune_valid(t) &&
            key == std::string(k).substr(0, std::string(k).find_last_not_of(' ') + 1)) {
          ctx->tune = t;
          found = true;
        }
      }
      fclose(f);
    }
  }
  int rc;
  if (!found) {
    if ((rc = forces_impl(ctx, true))) return rc;                // lists and bond data to time on
    if (ctx->fp64) tune_all<double>(ctx);
    else tune_all<float>(ctx);
    CK(cudaStreamSynchronize(ctx->st));
    ctx->forces_valid = false;                                  // the timing runs accumulated
    if ((rc = forces_impl(ctx, true))) return rc;
    if (cache_path) {
      if (FILE* f = fopen(cache_path, "a")) {
        const rx::Tune& t = ctx->tune;
        fprintf(f, "reaxff-tune %s | tors=%d nb=%d cf=%d bl=%d ang=%d hb=%d angl=%d qov=%d\n", key.c_str(),
                t.tors_lanes, t.nb_block, t.cf_block, t.bl_block, t.ang_block, t.hb_block, t.ang_lanes,
                t.qeq_overlap);
        fclose(f);
      }
    }
  }
  drop_graph(ctx);                                              // schedules are baked into the graph
  if (schedule) {
    const rx::Tune& t = ctx->tune;
    const int v[8] = {t.tors_lanes, t.nb_block, t.cf_block, t.bl_block, t.ang_block, t.hb_block, t.ang_lanes,
                      t.qeq_overlap};
    for (int q = 0; q < 8; ++q) schedule[q] = v[q];
  }
  return REAXFF_OK;
}

}  // extern "C"

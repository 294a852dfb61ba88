/*
 * reaxff.h -- C ABI of the GB300 (sm_103a) ReaxFF timestep library (libreaxff.so).
 *
 * One ReaxFF molecular-dynamics timestep (paper Sec. 2.1 and Fig. 1: bonded,
 * non-bonded and charge-equilibration interactions summed into per-atom forces)
 * runs here as hand-written CUDA kernels on one GPU:
 *   (a) cell-binned far-neighbour list, bond list and hydrogen-bond list (Sec. 3.3,
 *       "Neighbor and Interaction Lists"; Table 2 "Write Lists" / "Init. Forces"),
 *   (b) uncorrected -> corrected bond orders (Sec. 3.3 "Pairwise Interactions";
 *       Table 2 "Bond Orders"),
 *   (c) bonded terms: bond, lone pair, over/under-coordination, valence angle
 *       (+penalty, coalition), torsion (+conjugation), hydrogen bond (Sec. 2.1;
 *       Sec. 3.3 "Three-body Interactions"; Table 2 "3-body" / "4-body"),
 *   (d) tapered, shielded van der Waals and Coulomb terms (Sec. 3.3, Algorithm 2),
 *   (e) QEq: two Jacobi-preconditioned CG solves sharing the tapered H matrix,
 *       iterated concurrently (Sec. 3.3 "QEq"),
 *   (f) the dE/dBO chain rule into atom forces (Table 2 "Aggregate Forces") and
 *       velocity Verlet (Sec. 4.1: dt = 0.1 fs).
 *
 * Units: energy kcal/mol, length Angstrom, charge e, mass amu, time fs,
 *        force kcal/(mol A), velocity A/fs.
 * Boxes are orthorhombic and periodic; every box length must exceed r_nb.
 *
 * Ownership: every pointer argument is owned by the caller and only read or written
 * during the call. Host-pointer functions copy in/out; the context owns all device
 * memory it allocates. Functions suffixed _dev take device pointers and a
 * cudaStream_t (passed as void*) and enqueue work on that stream.
 *
 * Errors: every int-returning function returns REAXFF_OK (0) or a negative code;
 * reaxff_last_error() gives a text description. Nothing aborts the process.
 * The library is not thread-safe per context (one host thread per context).
 */
#ifndef REAXFF_H
#define REAXFF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REAXFF_MAXT 8       /* maximum number of atom types */
#define REAXFF_NTERMS 13    /* energy terms, in this order: */
/* 0 bond, 1 lp, 2 over, 3 under, 4 val, 5 pen, 6 coa, 7 tors, 8 conj, 9 hbond,
   10 vdw, 11 coul, 12 pol */

enum {
  REAXFF_OK = 0,
  REAXFF_E_INVALID = -1,        /* bad argument, parameter or size */
  REAXFF_E_CUDA = -2,           /* a CUDA runtime call failed (text has the CUDA error) */
  REAXFF_E_CAPACITY = -3,       /* a list overflowed even after the internal regrow */
  REAXFF_E_NOT_CONVERGED = -4,  /* QEq hit qeq_max_iter; charges still returned */
  REAXFF_E_TIMEOUT = -5,        /* a device-side wait hit its spin limit */
  REAXFF_E_NAN = -6,            /* non-finite positions, forces or energies */
  REAXFF_E_STATE = -7           /* call out of order (e.g. no positions set) */
};

enum { REAXFF_FP64 = 0, REAXFF_MIXED = 1 };                  /* options.precision */
/* options.warm_start: the QEq initial guess from the solutions of the previous steps (Sec. 3.3
 * names an extrapolation scheme without its form). The last 8 solutions of each system are
 * kept; a guess is sum_k w[m][k] x_k over the m kept (newest first), from one of three
 * predictors: 0, Lagrange (cubic through 4 points for s, quadratic through 3 for t); 1 and
 * 2, the value of the cubic fitted by least squares to the last 6 or 8 solutions (lower
 * degree while fewer are kept). The fits smooth the solve-tolerance noise of the stored
 * solutions, which dominates at loose tolerances; Lagrange has the smaller truncation error,
 * which dominates at tight ones. EXTRAP: adaptive, every solve scores the three predictors
 * against the solution it found and the best is used next, per replica and system;
 * LAGRANGE: predictor 0 always; ZERO: no history; MLP: EXTRAP plus the learned guess for s
 * (reaxff_mlp_*). */
enum { REAXFF_WARM_EXTRAP = 0, REAXFF_WARM_ZERO = 1, REAXFF_WARM_MLP = 2, REAXFF_WARM_LAGRANGE = 3 };
/* The weights of initial-guess predictor 0..2 (host only, no GPU): w (double[2*9*8])
 * receives w[sys][m][k], the weight of the k-th newest kept solution (k = 0 the newest)
 * when m are kept, for sys 0 (s) and 1 (t). E_INVALID for another predictor or a NULL w. */
int reaxff_extrap_weights(int32_t predictor, double* w);
/* options.qeq_precond: the CG preconditioner M of both QEq systems. JACOBI is the paper's
 * M = diag(H) (Sec. 3.3). BLOCK32 is block Jacobi over blocks of 32 consecutive atoms of a
 * replica (the last block of a replica may be shorter): M = blockdiag(H_BB), with each
 * block H_BB the exact restriction of H to the block (all images), inverted in FP32 once
 * per solve. Both run CG to the same tolerance; BLOCK32 needs fewer iterations when
 * strongly coupled atoms (molecules) are numbered consecutively. */
enum { REAXFF_PRECOND_JACOBI = 0, REAXFF_PRECOND_BLOCK32 = 1 };
enum { REAXFF_LIST_FAR = 0, REAXFF_LIST_BOND = 1, REAXFF_LIST_HBOND = 2 };

/* Force-field parameters (tables indexed by atom type). Per-pair tables are
 * symmetric; per-triple tables are [i][j=centre][k], symmetric in i<->k; torsion
 * tables are [j][k] for the central bond; H-bond tables are [X][Z] (X bonded to
 * the H atom, Z the acceptor). The functional forms that read them are listed in
 * each kernel's header comment. */
typedef struct {
  int32_t ntypes;
  int32_t hb[REAXFF_MAXT];          /* 0 none, 1 H-bond donor hydrogen, 2 acceptor */
  double mass[REAXFF_MAXT], val[REAXFF_MAXT], vale[REAXFF_MAXT], valboc[REAXFF_MAXT],
      valang[REAXFF_MAXT], p_lp2[REAXFF_MAXT], p_ovun2[REAXFF_MAXT], p_ovun5[REAXFF_MAXT],
      p_val3[REAXFF_MAXT], p_val5[REAXFF_MAXT], chi[REAXFF_MAXT], eta[REAXFF_MAXT],
      gamma_t[REAXFF_MAXT];
  double r0s[REAXFF_MAXT][REAXFF_MAXT], r0p[REAXFF_MAXT][REAXFF_MAXT],
      r0pp[REAXFF_MAXT][REAXFF_MAXT], p_bo1[REAXFF_MAXT][REAXFF_MAXT],
      p_bo2[REAXFF_MAXT][REAXFF_MAXT], p_bo3[REAXFF_MAXT][REAXFF_MAXT],
      p_bo4[REAXFF_MAXT][REAXFF_MAXT], p_bo5[REAXFF_MAXT][REAXFF_MAXT],
      p_bo6[REAXFF_MAXT][REAXFF_MAXT], p_boc3[REAXFF_MAXT][REAXFF_MAXT],
      p_boc4[REAXFF_MAXT][REAXFF_MAXT], p_boc5[REAXFF_MAXT][REAXFF_MAXT],
      ovc[REAXFF_MAXT][REAXFF_MAXT], v13[REAXFF_MAXT][REAXFF_MAXT],
      De_s[REAXFF_MAXT][REAXFF_MAXT], De_p[REAXFF_MAXT][REAXFF_MAXT],
      De_pp[REAXFF_MAXT][REAXFF_MAXT], p_be1[REAXFF_MAXT][REAXFF_MAXT],
      p_be2[REAXFF_MAXT][REAXFF_MAXT], p_ovun1[REAXFF_MAXT][REAXFF_MAXT],
      vdw_D[REAXFF_MAXT][REAXFF_MAXT], vdw_rv[REAXFF_MAXT][REAXFF_MAXT],
      vdw_alpha[REAXFF_MAXT][REAXFF_MAXT], vdw_gw[REAXFF_MAXT][REAXFF_MAXT],
      gamma[REAXFF_MAXT][REAXFF_MAXT];
  double th00[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT], p_val1[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT],
      p_val2[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT], p_val4[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT],
      p_val7[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT], p_pen1[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT],
      p_coa1[REAXFF_MAXT][REAXFF_MAXT][REAXFF_MAXT];
  double V1[REAXFF_MAXT][REAXFF_MAXT], V2[REAXFF_MAXT][REAXFF_MAXT], V3[REAXFF_MAXT][REAXFF_MAXT],
      p_tor1[REAXFF_MAXT][REAXFF_MAXT], p_cot1[REAXFF_MAXT][REAXFF_MAXT];
  double r0hb[REAXFF_MAXT][REAXFF_MAXT], p_hb1[REAXFF_MAXT][REAXFF_MAXT],
      p_hb2[REAXFF_MAXT][REAXFF_MAXT], p_hb3[REAXFF_MAXT][REAXFF_MAXT];
  double p_boc1, p_boc2, p_lp1, p_ovun3, p_ovun4, p_ovun6, p_ovun7, p_ovun8, p_val6, p_val8,
      p_val9, p_val10, p_pen2, p_pen3, p_pen4, p_coa2, p_coa3, p_coa4, p_tor2, p_tor3, p_tor4,
      p_cot2, p_vdW1, k_e;
} reaxff_params;

typedef struct {
  double r_nb;        /* nonbonded / QEq cutoff (A), 10 in the paper's setup (Sec. 4.2) */
  double r_bond;      /* bond-candidate cutoff (A) */
  double r_hb;        /* hydrogen-bond partner cutoff (A); r_bond <= r_hb <= r_nb */
  double bo_cut;      /* bond kept when BO'sig+BO'pi+BO'pp >= bo_cut */
  double thb_cut;     /* valence-angle / torsion bond-order threshold */
  double thb_cutsq;   /* valence-angle product threshold */
  double hb_bo_min;   /* minimum H-X bond order of an H-bond */
  double qeq_tol;     /* QEq relative residual ||b - Hx|| / ||b|| per system */
  int32_t qeq_max_iter;
  int32_t precision;  /* REAXFF_FP64 or REAXFF_MIXED (FP32 interaction math, FP64 sums) */
  int32_t warm_start; /* REAXFF_WARM_* */
  int32_t term_mask;  /* bit t set = energy term t contributes to forces (0 = all); bits
                         above the 13 terms select nothing, so 1 << 13 alone switches every
                         term off (free flight: zero forces, constant velocities) */
  double capacity_margin; /* list capacity headroom factor (>= 1; 0 = default 1.35) */
  double skin;        /* Verlet skin (A) of the neighbour candidate list, rebuilt on the device
                         only when an atom has moved more than skin/2; the far list is still
                         filtered exactly (r < r_nb) every step. 0 = default 0.7 A,
                         negative = no candidate list (cell stencil every step). A system
                         with a box edge <= r_nb + skin runs the cell stencil instead. */
  int32_t qeq_precond; /* REAXFF_PRECOND_* (0 = Jacobi) */
  int32_t spatial_sort; /* 1: the context stores the atoms of each replica in cell order
                           (5 A cells, z-major), taken from the positions of the first
                           reaxff_set_state and again at each reaxff_resort, for locality of
                           the neighbour gathers (Sec. 3.2's spatial ordering); every input and
                           output stays in the caller's order. 0: the caller's order. */
} reaxff_options;

typedef struct reaxff_ctx reaxff_ctx;

/* Layout checks for language bindings: sizes of the two structs and the byte offset
 * of a named field (returns -1 for an unknown name). */
int64_t reaxff_sizeof_params(void);
int64_t reaxff_sizeof_options(void);
int64_t reaxff_params_offset(const char* field);

/* Create a context for one periodic system of n atoms with the given types
 * (int32[n], each < params->ntypes) and box (double[3], A). Copies params and
 * options; allocates device memory sized from the density. *out receives the
 * context (NULL on error). */
int reaxff_create(const reaxff_params* params, const int32_t* types, int64_t n,
                  const double box[3], const reaxff_options* options, reaxff_ctx** out);

/* Create a context for nrep independent replicas (uneven sizes allowed) that run
 * together, one kernel launch per stage: replica r owns atoms
 * [rep_offsets[r], rep_offsets[r+1]) (int64[nrep+1], rep_offsets[0] = 0) and box
 * boxes[3r..3r+2]. No interaction crosses replicas; QEq and energies are per replica. */
int reaxff_create_batch(const reaxff_params* params, int32_t nrep, const int64_t* rep_offsets,
                        const int32_t* types, const double* boxes,
                        const reaxff_options* options, reaxff_ctx** out);

void reaxff_destroy(reaxff_ctx* ctx);
const char* reaxff_last_error(const reaxff_ctx* ctx);
int64_t reaxff_num_atoms(const reaxff_ctx* ctx);
int32_t reaxff_num_replicas(const reaxff_ctx* ctx);

/* Positions x (double[n*3], row-major xyz, A) and velocities v (double[n*3], A/fs,
 * NULL = zero). Positions are wrapped into [0, L). The QEq solution history used for
 * the extrapolated initial guess is kept (it only changes the starting point of CG,
 * never the converged charges); reaxff_reset_qeq_history() clears it. Positions equal
 * bit for bit to those the context holds (as last set or read back by get_state, with no
 * step since) keep the current forces, lists and candidate list, so a round trip of the
 * state through the host costs no extra force evaluation. */
int reaxff_set_state(reaxff_ctx* ctx, const double* x, const double* v);
/* With options.spatial_sort: store the atoms again in cell order of their current
 * positions (for long runs in which atoms wander away from their neighbours in memory). The
 * state is unchanged; the QEq solution history, bond-order averages and collected training
 * snapshots are dropped, and lists and forces are rebuilt at the next call. No-op without
 * spatial_sort. */
int reaxff_resort(reaxff_ctx* ctx);
/* Copy out positions, velocities (double[n*3]) and charges (double[n]); any may be NULL. */
int reaxff_get_state(reaxff_ctx* ctx, double* x, double* v, double* q);

/* (a) Build the far-neighbour, bond and H-bond lists for the current positions.
 * On overflow the library grows the list and rebuilds once; then E_CAPACITY. */
int reaxff_build_lists(reaxff_ctx* ctx);

/* Export a list built by reaxff_build_lists / reaxff_forces / reaxff_step in original
 * atom ids: entries (i[k], j[k], shift[3k..3k+2]) with the image shift s in {-1,0,1}^3
 * such that the neighbour is x_j + s*L. FAR and HBOND are directed (every ordered
 * pair), BOND is directed (both directions). capacity = length of i/j (shift has
 * 3*capacity); *count receives the entry count; E_INVALID if capacity < count
 * (*count is still set). Pass capacity 0 and NULL arrays to query the count. */
int reaxff_get_lists(reaxff_ctx* ctx, int32_t which, int64_t capacity, int64_t* count,
                     int32_t* i, int32_t* j, int8_t* shift);

/* (b) Bond orders of the directed bond list after reaxff_forces: per entry the
 * shifted uncorrected total BO' and the corrected BO, BO_pi, BO_pipi (double[count]),
 * in the order of reaxff_get_lists(BOND). Same capacity rules. */
int reaxff_get_bond_orders(reaxff_ctx* ctx, int64_t capacity, int64_t* count, double* bo_prime,
                           double* bo, double* bo_pi, double* bo_pipi);

/* (e) QEq at the current positions (builds lists): charges q (double[n] or NULL) and
 * CG iteration counts of the s and t systems (int32[nrep] each, or NULL). Returns
 * E_NOT_CONVERGED when a system hit qeq_max_iter (q is still written). */
int reaxff_qeq(reaxff_ctx* ctx, double* q_out, int32_t* iters_s, int32_t* iters_t);

/* (a)-(f) Forces at the current positions: lists, QEq, all terms, chain rule.
 * F: double[n*3]; E: double[nrep*13] per-replica energy terms; virial: double[nrep*6]
 * per replica, (xx, yy, zz, xy, xz, yz) of W_ab = -dE/d(strain_ab). Any may be NULL. */
int reaxff_forces(reaxff_ctx* ctx, double* F, double* E, double* virial);

/* Same with caller-fixed charges q (double[n]); QEq is skipped. */
int reaxff_forces_fixed_q(reaxff_ctx* ctx, const double* q, double* F, double* E,
                          double* virial);

/* nsteps velocity-Verlet steps of dt_fs (Sec. 4.1: dt = 0.1 fs). Each step updates the
 * lists, solves QEq and recomputes forces. E_tot (double[nsteps*nrep] or NULL) receives
 * the total (potential + kinetic) energy per step and replica.
 * The steps of one call run without host synchronisation (one CUDA graph per step where
 * stream capture is available); the device error flags are read once at the end. If a
 * list capacity overflowed anywhere in the call, the call is rolled back to its starting
 * positions, velocities and QEq history, the lists are regrown, and the steps are redone
 * with a check after every list build; the results are then the same as if the capacity
 * had been large enough from the start (up to the QEq history, which only moves the CG
 * starting point). Other errors (E_NAN, E_TIMEOUT, E_NOT_CONVERGED) are reported for
 * the call as a whole. */
int reaxff_step(reaxff_ctx* ctx, int32_t nsteps, double dt_fs, double* E_tot);

/* Kernel launches issued by the last reaxff_step call (for launch accounting). */
int64_t reaxff_last_launch_count(const reaxff_ctx* ctx);

/* CG iteration counts of the most recent QEq solve (int32[nrep] each, or NULL). */
int reaxff_last_qeq_iters(reaxff_ctx* ctx, int32_t* iters_s, int32_t* iters_t);

/* Forget the QEq solution history (the next solve starts from zero). */
void reaxff_reset_qeq_history(reaxff_ctx* ctx);

/* Limit, in SM clock cycles, of every wait of the persistent QEq kernel at its grid
 * barrier (Sec. 3.3's concurrent CG iterations synchronise there); cycles <= 0 restores
 * the default (3e9 cycles, about 1.5 s at 2 GHz). A wait that runs out sets the device
 * error flag and every block leaves the solve at its next barrier, so the call returns
 * REAXFF_E_TIMEOUT instead of waiting on; the context stays usable. A small limit is a
 * test hook for that path; the default is what production runs use. */
int reaxff_set_wait_limit(reaxff_ctx* ctx, int64_t cycles);

/* Per replica (int32[nrep]): 1 where the last QEq solve started s from the learned guess
 * (options.warm_start = REAXFF_WARM_MLP with a trained network), 0 where the extrapolated
 * guess had the smaller initial residual. */
int reaxff_qeq_warm_choice(reaxff_ctx* ctx, int32_t* mlp_used);

/* Sparse matrix-vector products (one read of H for both systems) performed by all QEq
 * solves of this context since its creation: the initial residual of every solve plus
 * one per CG iteration. Synchronises the context's stream; -1 on a CUDA error. */
int64_t reaxff_qeq_spmv_total(reaxff_ctx* ctx);

/* Per-stage timing with CUDA events recorded on the context's stream around every
 * kernel group (cells, far_list, bond_list, bo_prime64, qeq, bo_correct, atom_terms,
 * over_under_bond, s_gather, angles, torsions, hbonds, nonbonded, chain_rule, verlet,
 * reduce, mlp_guess, qeq_precond), the groups run one after another. enable(2) instead
 * keeps the QEq solve beside the charge-free terms (where the schedule has it there) and
 * times that part as two spans from the fork: solve_path (solve and nonbonded kernel) and
 * terms_path (bond list, bond orders, bonded terms, chain rule); the groups outside it are
 * timed as with enable(1). enable(0) turns timing off; enable(1 or 2) also zeroes the
 * totals. read() fills ms[] (accumulated milliseconds) and calls[] (timed launches) for up
 * to nstage stages and returns the number of stages; stage_name() gives each stage's name. */
void reaxff_profile_enable(reaxff_ctx* ctx, int32_t on);
int32_t reaxff_profile_read(reaxff_ctx* ctx, int32_t nstage, double* ms, int64_t* calls);
const char* reaxff_stage_name(int32_t stage);

/* ---- device-pointer variants (no host copies; enqueue on `stream`) ---------------- */
int reaxff_set_state_dev(reaxff_ctx* ctx, const double* x_dev, const double* v_dev, void* stream);
int reaxff_get_state_dev(reaxff_ctx* ctx, double* x_dev, double* v_dev, double* q_dev, void* stream);
/* Runs nsteps on `stream`; no host synchronisation unless a list overflows.
 * E_tot_dev: double[nsteps*nrep] on the device, or NULL. */
int reaxff_step_dev(reaxff_ctx* ctx, int32_t nsteps, double dt_fs, double* E_tot_dev, void* stream);

/* ---- allocation-free far-list builder ----------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory while they run: applications that hand out all GPU memory
 * from their own pool and forbid runtime allocation, latency-bound loops where the
 * device-wide synchronisation of cudaMalloc/cudaFree would stall other work, and
 * plug-ins whose host framework must account for every allocation. It builds the same
 * cell-binned far-neighbour list and QEq H entries as reaxff_build_lists (FP64 path)
 * for one periodic system, without a context and without allocating: its scratch (cell
 * grid, FP32 position copies, sorted atoms, parameter block; about 2.9 MB) is one
 * file-scope __device__ array that every GPU loading the library keeps until exit.
 *
 * Limits: n <= 65536 atoms, at most 16384 cells (cell edge >= r_nb) and n * cap below
 * 2^31 entries; larger inputs are rejected with REAXFF_E_INVALID. Inputs (device
 * pointers): types int32[n], each in [0, ntypes), and positions x, y, z double[n] each,
 * already wrapped into [0, L); a device-side check runs first, and a type or position
 * outside those ranges (or not finite) returns REAXFF_E_INVALID with no list built. Outputs (device
 * pointers, caller-allocated): cnt int32[n] (entries per row, at most cap),
 * j int32[n*cap] and shift uint8[n*cap] (image code (sx+1)*9 + (sy+1)*3 + (sz+1)) and
 * H double[n*cap], row i at [i*cap, i*cap + cnt[i]). Returns REAXFF_E_CAPACITY when a
 * row had more than cap neighbours (that row is truncated). params/options and box are
 * host pointers. Work is enqueued on `stream`; the call waits for it to finish.
 * *err_msg (if not NULL) receives a static description of any error.
 * No call can be captured into a CUDA graph: each one reads its error flags back to the
 * host and waits for the stream. The first call on each device also looks up the scratch
 * array's device address (once per device, with that device current).
 * The address is kept for the life of the process, so the entry point must not be used
 * on a device after cudaDeviceReset (a new context would not hold that address).
 * All calls share the one scratch array and each call clears what must start at zero;
 * calls that overlap on the GPU (several streams or host threads) race on it. */
int reaxff_far_list_noalloc(const reaxff_params* params, const reaxff_options* options,
                            const int32_t* types_dev, const double* x_dev, const double* y_dev,
                            const double* z_dev, int64_t n, const double box[3], int32_t cap,
                            int32_t* cnt_dev, int32_t* j_dev, uint8_t* shift_dev, double* H_dev,
                            void* stream, const char** err_msg);

/* ---- (e5) Learned QEq warm start -------------------------------------------------------
 * Sec. 3.3 starts the QEq CG from an extrapolated guess; a per-atom network trained on
 * charges the method itself produced gives another guess (options.warm_start =
 * REAXFF_WARM_MLP). CG still runs to the same tolerance, so the guess moves only its
 * starting point. Descriptors: REAXFF_MLP_NF = 192 per atom, for each neighbour element
 * e = 0..3 (element types must be 0..3): 32 radial Gaussians sum exp(-eta (r - mu_k)^2)
 * fc(r) (mu_k = 0.8 + 5.2 k/31 A, eta = 1/(2 (5.2/31)^2), cosine cutoff 6 A) and 16
 * angular terms 2^(1-zeta) sum over ordered neighbour pairs (j of e, k any, both within
 * 3.5 A) of (1 + lambda cos theta)^zeta exp(-eta_a (r_ij^2 + r_ik^2)) fc fc, zeta in
 * {1,2,4,8}, eta_a in {0.05, 0.3}, lambda in {+1,-1}, index 4 zeta_idx + 2 eta_idx +
 * lambda_idx; per element [32 radial, 16 angular]. Network per centre element:
 * x~ = (x - mean) inv_std, z1 = x~ W1 + b1, z2 = silu(z1) W2 + b2, y = silu(z2) . w3 + b3
 * (192 -> 64 -> 64 -> 1). Parameters per element (float, REAXFF_MLP_NPAR = 16577):
 * W1[192][64] row-major, b1[64], W2[64][64], b2[64], w3[64], b3; four elements in a row.
 * Inference runs BF16 operands on the tensor cores with FP32 accumulation; training runs
 * FP32 kernels (MSE loss over the atoms of one snapshot per Adam step). All buffers are
 * host pointers; every call synchronises the context's stream. */
#define REAXFF_MLP_NF 192
#define REAXFF_MLP_NPAR 16577
/* Seeded initial parameters (normal, variance 1/fan-in; biases 0; the output biases are
 * set to the mean training charge of each element by the first reaxff_mlp_train). */
int reaxff_mlp_init(reaxff_ctx* ctx, uint64_t seed);
/* Parameters theta float[4*16577], normalisation mean float[192] and inv_std float[192]
 * (0 for a constant feature); set marks the network ready for prediction. */
int reaxff_mlp_set_params(reaxff_ctx* ctx, const float* theta, const float* mean, const float* inv_std);
int reaxff_mlp_get_params(reaxff_ctx* ctx, float* theta, float* mean, float* inv_std);
/* Descriptors float[n*192] of the current positions (lists built if needed).
 * E_CAPACITY if an atom has more than 192 neighbours within 6 A or 64 within 3.5 A. */
int reaxff_mlp_descriptors(reaxff_ctx* ctx, float* D);
/* Tensor-core forward of the context's network on m caller descriptor rows
 * (float[m*192], raw, normalised inside) of elements types int32[m]; y float[m]. */
int reaxff_mlp_infer(reaxff_ctx* ctx, const float* D, const int32_t* types, int64_t m, float* y);
/* FP32 loss L = mean_i (y_i - q_i)^2 over m caller rows and dL/dtheta float[4*16577]. */
int reaxff_mlp_loss_grad(reaxff_ctx* ctx, const float* D, const int32_t* types, const float* q, int64_t m,
                         float* grad, double* loss);
/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step counter kept
 * by the context) of the parameters with the caller's gradient float[4*16577]. */
int reaxff_mlp_adam_step(reaxff_ctx* ctx, const float* grad, double lr);
/* Training set of nsnap snapshots (descriptors and charges of all atoms); clears it. */
int reaxff_mlp_reserve(reaxff_ctx* ctx, int32_t nsnap);
/* Append the current state (its descriptors and QEq charges; forces are computed first
 * if the current positions have none) to the training set. E_CAPACITY when full. */
int reaxff_mlp_collect(reaxff_ctx* ctx);
/* epochs passes over the collected snapshots in order, one Adam step (learning rate lr)
 * per snapshot; normalisation statistics from the whole set; loss_out (or NULL) gets
 * the mean loss of the last pass. The network is then ready. */
int reaxff_mlp_train(reaxff_ctx* ctx, int32_t epochs, double lr, double* loss_out);
/* Predicted charges double[n] at the current positions (tensor-core inference). */
int reaxff_mlp_predict(reaxff_ctx* ctx, double* q);

/* ---- In-situ molecular species analysis (Sec. 3.4) ----------------------------------------
 * At the current positions (forces are computed first if the current positions have none):
 * atoms i, j are bonded when their corrected bond order exceeds bo_threshold[t_i*8 + t_j]
 * (double[REAXFF_MAXT*REAXFF_MAXT], or NULL for 0.3 everywhere); a molecule is a connected
 * component of that graph, numbered 0..M-1 in the order of its smallest atom index; a
 * species is the vector of atom counts per type of a molecule (isomers not told apart).
 * mol_id (int32[n] or NULL) receives each atom's molecule, *nmol (or NULL) M. species
 * (int32[cap][REAXFF_MAXT + 2], rows: replica, count of type 0..7, molecules) receives the
 * summary sorted by (replica, counts) and *nspecies its length; E_CAPACITY (with
 * *nspecies set) when it has more than cap rows. Connectivity, numbering and counting run
 * on the GPU; the host tallies the M count vectors into the summary. */
int reaxff_species(reaxff_ctx* ctx, const double* bo_threshold, int32_t* mol_id, int64_t* nmol, int32_t cap,
                   int32_t* species, int32_t* nspecies);

/* Time-averaged bonds (Sec. 3.4: persistent bonds told from transient encounters by
 * averaging bond orders over samples). reaxff_bo_average_sample adds the corrected bond
 * order of every directed bond-list entry at the current positions (forces computed first
 * when stale) to a running sum kept per (atom, neighbour, image); a pair missing from a
 * sample adds 0, so the average is sum / samples over all samples taken since the last
 * reset. Device work only, no synchronisation. reaxff_bo_average_reset clears the sums
 * (also before the first sample). reaxff_get_bo_average exports every pair seen, directed,
 * with its average (arrays as reaxff_get_lists plus avg double[count]; same capacity
 * rules). reaxff_species_average runs reaxff_species's analysis with the averages in place
 * of the instantaneous bond orders (same arguments and outputs). E_STATE without samples;
 * E_CAPACITY when an atom met more distinct bonded pairs than its row holds (2 x the bond
 * capacity, at least 48). */
int reaxff_bo_average_reset(reaxff_ctx* ctx);
int reaxff_bo_average_sample(reaxff_ctx* ctx);
int64_t reaxff_bo_average_samples(reaxff_ctx* ctx);
int reaxff_get_bo_average(reaxff_ctx* ctx, int64_t capacity, int64_t* count, int32_t* i, int32_t* j,
                          int8_t* shift, double* avg);
int reaxff_species_average(reaxff_ctx* ctx, const double* bo_threshold, int32_t* mol_id, int64_t* nmol,
                           int32_t cap, int32_t* species, int32_t* nspecies);

/* ---- Launch-schedule autotuner ----------------------------------------------------------
 * Times the alternatives of each tunable launch schedule on this context's current data
 * with CUDA events and keeps the fastest:
 *  - lanes per central bond in the torsion kernel (2, 4, 8);
 *  - lanes per centre atom in the angle kernel (8, 16, 32; mixed path);
 *  - threads per block of the nonbonded, candidate-filter, bond-list, angle and H-bond
 *    kernels;
 *  - (mixed path) where the QEq solve runs. 0: before the charge-independent bond-order
 *    and bonded terms. On a second stream beside them: 1 / 2 with a half / a quarter of every
 *    SM's threads; 3 / 4 / 5 with 1024-thread blocks on 1/2, 3/8 or 5/8 of the SMs. This entry is timed on MD steps (0.1 fs, from the context's state,
 *    which is restored afterwards). The results agree to within the rounding of the CG dot
 *    products, whose partial sums follow the thread count and the rows per block.
 * With the solve beside the terms, the torsion lanes (1, 2, 4, 8), angle lanes (4, 8, 16,
 * 32), angle, H-bond, nonbonded and bond-list blocks are timed again by whole force
 * evaluations in that schedule. Needs positions; forces are recomputed afterwards (the
 * timing runs accumulate into them).
 * cache_path (or NULL): a text file of "reaxff-tune <key> | ..." lines, the key being (n,
 * replicas, precision, skin, compute capability, SM count). A matching line whose every entry
 * is one the tuner can pick is used instead of timing; otherwise the context is tuned and
 * the result appended.
 * schedule (int32[8] or NULL) receives (torsion lanes, nonbonded, filter, bond list, angles,
 * H-bonds, angle lanes, QEq placement 0..5). */
int reaxff_autotune(reaxff_ctx* ctx, const char* cache_path, int32_t* schedule);

#ifdef __cplusplus
}
#endif
#endif /* REAXFF_H */

// In-situ molecular species analysis (Sec. 3.4).
//
// Two atoms are bonded when their corrected bond order exceeds a threshold for the pair
// of elements (default 0.3). The molecule of an atom is its connected component in that
// bond graph, identified by the smallest atom index in it; molecules are numbered
// 0..M-1 in the order of those indices; a species is the vector of atom counts per
// element of a molecule (isomers are not distinguished), and the summary counts the
// molecules of each species.
//
// GPU form: every atom starts as its own root (label = index). A hooking pass visits each
// bond above the threshold once (j > i) and hooks the larger of the two endpoint roots
// under the smaller one with atomicMin; a compression pass points every atom at its root.
// Labels only decrease and always point to a smaller or equal index, so root walks end,
// and the fixed point -- every component labelled by its minimum index -- does not depend
// on the order of the atomics. Passes repeat until no hook happens (host loop on a device
// flag). Roots are ranked by a two-level prefix count, atoms take their root's rank, and
// per-molecule element counts are integer atomics.
#include "reax_internal.cuh"

namespace {

__device__ __forceinline__ int find_root(const int* lab, int a) {
  int b = lab[a];
  while (b != a) {
    a = b;
    b = lab[a];
  }
  return a;
}

__global__ void k_sp_init(int* lab, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lab[i] = i;
}

template <typename R>
__global__ void k_sp_hook(Sys s, BondList bl, const R* bo, const double* thr, int* lab, int* changed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int ti = s.type[i];
  const int nb = bl.cnt[i];
  for (int k = 0; k < nb; ++k) {
    const int e = i * bl.cap + k;
    const int j = bl.j[e];
    if (j <= i) continue;                               // each bond once, self-images skipped
    if (!((double)bo[e] > thr[ti * MAXT + s.type[j]])) continue;
    const int a = find_root(lab, i), b = find_root(lab, j);
    if (a != b) {
      atomicMin(lab + max(a, b), min(a, b));
      *changed = 1;
    }
  }
}

__global__ void k_sp_compress(int* lab, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lab[i] = find_root(lab, i);
}

constexpr int SP_BLOCK = 1024;

// roots per block of SP_BLOCK atoms
__global__ void k_sp_blockcount(const int* lab, int n, int* bcount) {
  const int i = blockIdx.x * SP_BLOCK + threadIdx.x;
  const int r = (i < n && lab[i] == i) ? 1 : 0;
  const int c = __syncthreads_count(r);
  if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

// exclusive prefix of the block counts (one thread; at most n / 1024 values) and M
__global__ void k_sp_scanblocks(int* bcount, int nb, int* total) {
  int run = 0;
  for (int b = 0; b < nb; ++b) {
    const int c = bcount[b];
    bcount[b] = run;
    run += c;
  }
  *total = run;
}

// rank of every root among the roots (by index)
__global__ void k_sp_rank(const int* lab, int n, const int* boff, int* rank) {
  __shared__ int wsum[SP_BLOCK / 32];
  const int i = blockIdx.x * SP_BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool r = i < n && lab[i] == i;
  const unsigned m = __ballot_sync(0xffffffffu, r);
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int before = 0;
  for (int q = 0; q < w; ++q) before += wsum[q];
  if (r) rank[i] = boff[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u));
}

__global__ void k_sp_count(Sys s, const int* lab, const int* rank, int* mol, int* cnt, int* mrep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int m = rank[lab[i]];
  mol[i] = m;
  atomicAdd(cnt + (size_t)m * MAXT + s.type[i], 1);
  mrep[m] = s.rep[i];                                   // every atom of a molecule: same replica
}

// Time-averaged bond orders (Sec. 3.4: bonds decided from bond orders averaged over samples
// rather than one instant). One thread per atom adds each bond entry's corrected BO to the
// running sum of the same (neighbour, image) in the atom's row, appending the pair when it
// is new; a pair absent from a sample adds nothing, so sum / samples is the average with
// zeros for the samples without it. Each row is owned by one thread and samples are added
// in order: deterministic. The two directions of a bond carry the same BO in every sample,
// so their sums are equal.
template <typename R>
__global__ void k_boavg_sample(Sys s, BondList bl, rx::BoAvg A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const R* bo = (const R*)bl.bo;
  const size_t row = (size_t)i * A.cap;
  int m = A.cnt[i];
  const int nb = bl.cnt[i];
  for (int k = 0; k < nb; ++k) {
    const size_t e = (size_t)i * bl.cap + k;
    const int j = bl.j[e];
    const uint8_t c = bl.s[e];
    const double v = (double)bo[e];
    int q = 0;
    while (q < m && !(A.j[row + q] == j && A.s[row + q] == c)) ++q;
    if (q < m) {
      A.sum[row + q] += v;
    } else if (m < A.cap) {
      A.j[row + m] = j;
      A.s[row + m] = c;
      A.sum[row + m] = v;
      ++m;
    } else {
      *A.over = 1;
    }
  }
  A.cnt[i] = m;
}

__global__ void k_boavg_finish(int n, rx::BoAvg A, double inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t row = (size_t)i * A.cap;
  for (int q = 0; q < A.cnt[i]; ++q) A.avg[row + q] = A.sum[row + q] * inv;
}

}  // namespace

namespace rx {

template <typename R>
void bo_average_sample(const Launch& L, Sys s, BondList bl, BoAvg A) {
  k_boavg_sample<R><<<(s.n + 127) / 128, 128, 0, L.st>>>(s, bl, A);
  *L.count += 1;
}

void bo_average_finish(const Launch& L, int n, BoAvg A, double inv_samples) {
  k_boavg_finish<<<(n + 255) / 256, 256, 0, L.st>>>(n, A, inv_samples);
  *L.count += 1;
}

template void bo_average_sample<double>(const Launch&, Sys, BondList, BoAvg);
template void bo_average_sample<float>(const Launch&, Sys, BondList, BoAvg);

// labels to the component minima; returns the number of hooking passes, or -1 when the
// pass limit was reached (flags read on the host: synchronises the stream)
template <typename R>
int species_components(const Launch& L, Sys s, BondList bl, const double* thr, SpeciesBuf& b, int max_pass) {
  const int g = (s.n + 255) / 256;
  k_sp_init<<<g, 256, 0, L.st>>>(b.lab, s.n);
  *L.count += 1;
  for (int pass = 1; pass <= max_pass; ++pass) {
    cudaMemsetAsync(b.changed, 0, sizeof(int), L.st);
    k_sp_hook<R><<<g, 256, 0, L.st>>>(s, bl, (const R*)bl.bo, thr, b.lab, b.changed);
    k_sp_compress<<<g, 256, 0, L.st>>>(b.lab, s.n);
    *L.count += 2;
    int h = 1;
    cudaMemcpyAsync(b.h_changed, b.changed, sizeof(int), cudaMemcpyDeviceToHost, L.st);
    cudaStreamSynchronize(L.st);
    h = *b.h_changed;
    if (!h) return pass;
  }
  return -1;
}

void species_molecules(const Launch& L, Sys s, SpeciesBuf& b) {
  const int nb = (s.n + SP_BLOCK - 1) / SP_BLOCK;
  k_sp_blockcount<<<nb, SP_BLOCK, 0, L.st>>>(b.lab, s.n, b.boff);
  k_sp_scanblocks<<<1, 1, 0, L.st>>>(b.boff, nb, b.nmol);
  k_sp_rank<<<nb, SP_BLOCK, 0, L.st>>>(b.lab, s.n, b.boff, b.rank);
  cudaMemsetAsync(b.cnt, 0, (size_t)s.n * MAXT * sizeof(int), L.st);
  k_sp_count<<<(s.n + 255) / 256, 256, 0, L.st>>>(s, b.lab, b.rank, b.mol, b.cnt, b.mrep);
  *L.count += 4;
}

template int species_components<double>(const Launch&, Sys, BondList, const double*, SpeciesBuf&, int);
template int species_components<float>(const Launch&, Sys, BondList, const double*, SpeciesBuf&, int);

}  // namespace rx

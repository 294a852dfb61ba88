// Allocation-free far-neighbour list builder (see reaxff_far_list_noalloc in reaxff.h).
//
// For callers that must not allocate device memory while they run: everything this
// entry point needs beyond the caller's inputs and outputs lives in one file-scope
// __device__ array of fixed size, so it issues no cudaMalloc / cudaFree and uses no
// allocating library routine. The array is shared by every call in the process and
// keeps the previous call's contents; the counters that must start at zero are cleared
// by each call. Calls that overlap on the GPU (other streams, other host threads) race
// on the array.
#include <cstring>

#include "reax_internal.cuh"

namespace {

constexpr int NOALLOC_MAX_ATOMS = 65536;
constexpr int NOALLOC_MAX_CELLS = 16384;
constexpr int NOALLOC_MAX_DEVICES = 64;

// layout of the scratch array (header first, then the per-atom and per-cell arrays)
struct Header {
  DParams<double> P;
  double box[3];
  int64_t rep_off[2];
  float boxh[3], boxl[3];
  int nc[3];
  int cell_off[2];
  int err;
};
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t OFF_XH = align256(sizeof(Header));
constexpr size_t FLT_BYTES = align256(sizeof(float) * NOALLOC_MAX_ATOMS);
constexpr size_t INT_BYTES = align256(sizeof(int) * NOALLOC_MAX_ATOMS);
constexpr size_t CELL_BYTES = align256(sizeof(int) * (NOALLOC_MAX_CELLS + 1));
constexpr size_t OFF_INT = OFF_XH + 6 * FLT_BYTES;           // xh yh zh xl yl zl
constexpr size_t OFF_CELL = OFF_INT + 4 * INT_BYTES;          // rep atom_cell atoms tmp
constexpr size_t SCRATCH_BYTES = OFF_CELL + 3 * CELL_BYTES;   // count start cursor (~2.9 MB)

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

unsigned char* g_scratch_dev[NOALLOC_MAX_DEVICES] = {nullptr};

// input-check bits of this entry point (kept apart from the list kernels' bits)
constexpr int NOALLOC_BAD_TYPE = 1 << 20;
constexpr int NOALLOC_BAD_POS = 1 << 21;

// Device-side input check, run before any kernel indexes a table by type or a cell by
// position: a type outside [0, ntypes) would index the per-pair tables out of range, and a
// position outside [0, L) (or not finite) would be clamped into an edge cell, where the
// 27-cell stencil misses some of its neighbours.
__global__ void k_noalloc_check(const int32_t* __restrict__ type, const double* __restrict__ x,
                                const double* __restrict__ y, const double* __restrict__ z, int n,
                                int ntypes, double Lx, double Ly, double Lz, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int bad = 0;
  int t = type[i];
  if (t < 0 || t >= ntypes) bad |= NOALLOC_BAD_TYPE;
  double p[3] = {x[i], y[i], z[i]};
  double L[3] = {Lx, Ly, Lz};
  for (int d = 0; d < 3; ++d)
    if (!(p[d] >= 0.0 && p[d] < L[d])) bad |= NOALLOC_BAD_POS;   // also catches NaN
  if (bad) atomicOr(err, bad);
}

}  // namespace

void rx_fill_params_double(DParams<double>& d, const reaxff_params& p, const reaxff_options& o);

extern "C" int reaxff_far_list_noalloc(const reaxff_params* params, const reaxff_options* options,
                                       const int32_t* types_dev, const double* x_dev, const double* y_dev,
                                       const double* z_dev, int64_t n, const double box[3], int32_t cap,
                                       int32_t* cnt_dev, int32_t* j_dev, uint8_t* shift_dev, double* H_dev,
                                       void* stream, const char** err_msg) {
  const char* dummy = nullptr;
  const char** em = err_msg ? err_msg : &dummy;
  *em = "";
  if (!params || !options || !types_dev || !x_dev || !y_dev || !z_dev || !box || !cnt_dev || !j_dev ||
      !shift_dev || !H_dev) {
    *em = "null argument";
    return REAXFF_E_INVALID;
  }
  if (n < 1 || n > NOALLOC_MAX_ATOMS) {
    *em = "n out of range: the allocation-free list builder holds at most 65536 atoms";
    return REAXFF_E_INVALID;
  }
  if (cap < 1 || params->ntypes < 1 || params->ntypes > MAXT || !(options->r_nb > 0)) {
    *em = "invalid cap, ntypes or r_nb";
    return REAXFF_E_INVALID;
  }
  if ((int64_t)n * (int64_t)cap > (int64_t)INT32_MAX) {
    *em = "n * cap exceeds 2^31 - 1 entries (row offsets are 32-bit)";
    return REAXFF_E_INVALID;
  }
  int nc[3], ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > options->r_nb)) {
      *em = "every box length must exceed r_nb";
      return REAXFF_E_INVALID;
    }
    nc[d] = (int)std::floor(box[d] / options->r_nb);
    if (nc[d] < 1) nc[d] = 1;
    ncell *= nc[d];
    if (ncell > NOALLOC_MAX_CELLS) break;
  }
  if (ncell > NOALLOC_MAX_CELLS) {
    *em = "box too large: the allocation-free list builder holds at most 16384 cells";
    return REAXFF_E_INVALID;
  }
  // once per device: the device address of the scratch array (host code only has a
  // host-side stand-in for the symbol)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    *em = "cudaGetDevice failed or device index too large";
    return REAXFF_E_CUDA;
  }
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *em = "cudaGetSymbolAddress of the scratch array failed";
      return REAXFF_E_CUDA;
    }
    g_scratch_dev[dev] = (unsigned char*)p;
  }
  unsigned char* base = g_scratch_dev[dev];
  cudaStream_t st = (cudaStream_t)stream;
  // header (parameters, box, cell grid) from the host
  Header h;
  memset(&h, 0, sizeof(h));
  rx_fill_params_double(h.P, *params, *options);
  double lmax = 0;
  for (int d = 0; d < 3; ++d) {
    h.box[d] = box[d];
    h.boxh[d] = (float)box[d];
    h.boxl[d] = (float)(box[d] - (double)h.boxh[d]);
    h.nc[d] = nc[d];
    lmax = box[d] > lmax ? box[d] : lmax;
  }
  h.rep_off[0] = 0;
  h.rep_off[1] = n;
  h.cell_off[0] = 0;
  h.cell_off[1] = ncell;
  h.err = 0;
  Header* hd = (Header*)base;
  float* fl = (float*)(base + OFF_XH);
  int* in = (int*)(base + OFF_INT);
  int* ce = (int*)(base + OFF_CELL);
  auto F = [&](int k) { return (float*)((unsigned char*)fl + k * FLT_BYTES); };
  auto I = [&](int k) { return (int*)((unsigned char*)in + k * INT_BYTES); };
  auto Cc = [&](int k) { return (int*)((unsigned char*)ce + k * CELL_BYTES); };
  cudaError_t e = cudaMemcpyAsync(hd, &h, sizeof(Header), cudaMemcpyHostToDevice, st);
  // every atom belongs to replica 0: clear the replica ids the previous call left
  if (e == cudaSuccess) e = cudaMemsetAsync(I(0), 0, sizeof(int) * n, st);
  if (e != cudaSuccess) {
    *em = "copy of the header into the scratch array failed";
    return REAXFF_E_CUDA;
  }
  // reject invalid device inputs before any kernel uses them as indexes
  int flags = 0;
  k_noalloc_check<<<(int)((n + 255) / 256), 256, 0, st>>>(types_dev, x_dev, y_dev, z_dev, (int)n,
                                                          params->ntypes, box[0], box[1], box[2], &hd->err);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, &hd->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    *em = "input check launch or synchronisation failed";
    return REAXFF_E_CUDA;
  }
  if (flags & NOALLOC_BAD_TYPE) {
    *em = "a type is outside [0, ntypes)";
    return REAXFF_E_INVALID;
  }
  if (flags & NOALLOC_BAD_POS) {
    *em = "a position is outside [0, L) or not finite (wrap positions into the box first)";
    return REAXFF_E_INVALID;
  }
  Sys s{};
  s.n = (int)n;
  s.nrep = 1;
  s.type = types_dev;
  s.rep = I(0);
  s.box = hd->box;
  s.rep_off = hd->rep_off;
  s.boxh = hd->boxh;
  s.boxl = hd->boxl;
  s.x = const_cast<double*>(x_dev);
  s.y = const_cast<double*>(y_dev);
  s.z = const_cast<double*>(z_dev);
  s.xh = F(0); s.yh = F(1); s.zh = F(2);
  s.xl = F(3); s.yl = F(4); s.zl = F(5);
  s.err = &hd->err;
  Cells c{};
  c.nc = hd->nc;
  c.cell_off = hd->cell_off;
  c.ncell_total = ncell;
  c.count = Cc(0);
  c.start = Cc(1);
  c.cursor = Cc(2);
  c.atom_cell = I(1);
  c.atoms = I(2);
  c.tmp = I(3);
  c.slices = 1;
  FarList f{};
  f.cap = cap;
  f.cnt = cnt_dev;
  f.j = j_dev;
  f.s = shift_dev;
  f.H = H_dev;
  const double u = std::ldexp(1.0, -24);
  const float margin = (float)(32.0 * u * (lmax * options->r_nb + options->r_nb * options->r_nb));
  int64_t launches = 0;
  rx::Launch L{st, &launches};
  rx::cells_build(L, s, c);
  rx::far_list<double>(L, s, c, f, &hd->P, margin);
  flags = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, &hd->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    *em = "kernel launch or synchronisation failed";
    return REAXFF_E_CUDA;
  }
  if (flags & ERR_CAP_FAR) {
    *em = "a row has more neighbours than cap (rows are truncated to cap)";
    return REAXFF_E_CAPACITY;
  }
  return REAXFF_OK;
}

// The C ABI of liblbm_gb300.so (declared and documented in include/lbm_gb300.h):
// handle lifecycle, device memory through the allocator hook, geometry set-up,
// state conversion, the time loop (replayed from CUDA graphs) and readback.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "lbm_model.cuh"

using namespace lbm;

namespace {

thread_local std::string g_error;

std::mutex g_alloc_mu;
lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

constexpr int kGraphSteps = 16;   // steps per captured graph (even: parity returns)

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

struct Lattice {
  lbm_desc desc{};
  int64_t N = 0, nf = 0, nstore = 0, stride = 0;
  uint8_t* flags = nullptr;
  void* pdf[2] = {nullptr, nullptr};
  uint32_t* link = nullptr;   // [18][stride] element offsets (see LatticeView)
  int32_t* cell_of = nullptr;
  int32_t* list_index = nullptr;
  int* status = nullptr;   // the handle's device status word
  // run-indexed code of `link` (lbm_ria.cu), indirect lattices only
  uint2* ria_head = nullptr;
  uint32_t* ria_pool = nullptr;
  uint32_t* ria_chunk_start = nullptr;
  int64_t ria_pool_entries = 0;
  bool has_halfway = false, has_fullway = false;
  bool geometry = false, params = false, init = false;
  double omega = 1.0, Lambda = 0.25;
  TrtParams trt;

  bool indirect() const { return desc.addressing == LBM_INDIRECT; }
  LatticeView view() const {
    LatticeView v;
    v.nx = desc.nx;
    v.ny = desc.ny;
    v.nz = desc.nz;
    v.n_cells = N;
    v.n_nodes = nstore;
    v.stride = stride;
    v.prec = desc.precision;
    v.indirect = indirect();
    v.has_halfway = has_halfway;
    v.flags = flags;
    v.link = link;
    v.cell_of = cell_of;
    v.list_index = list_index;
    v.status = status;
    return v;
  }
};

}  // namespace

struct lbm_lattice_s {
  std::vector<Lattice> lat;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  int prec = 0, prop = 0;
  int64_t steps = 0;     // since the last init / write
  int phase = 0;         // total steps mod 2: AA parity, pull buffer holding the state
  bool poisoned = false;
  int threads = 256, cells_per_thread = 1, ctas_per_sm = 0;
  bool run_indexing = true;   // staged list sweeps read the run-indexed links
  int steps_per_pass = 1;     // 2: temporal blocking (single full-array pull lattice)
  bool two_step() const {
    return steps_per_pass == 2 && lat.size() == 1 && prop == LBM_PULL_TWO_GRID && !lat[0].indirect();
  }
  // batch work list: one descriptor per lattice and the tiles (rebuilt lazily)
  void* d_lat = nullptr;
  size_t d_lat_bytes = 0;
  BatchTile* d_tiles = nullptr;
  size_t d_tiles_bytes = 0;
  int ntiles = 0;
  bool tables_dirty = true;
  bool batched() const { return lat.size() > 1; }
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn free_ = nullptr;
  void* alloc_ctx = nullptr;
  int64_t bytes = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int* d_status = nullptr;   // kernels set bits here (bounded waits that gave up)
  // FP16 stochastic format: the seed of lattice 0 (lattice l uses seed + l) and
  // the pair of sweep counters; word `phase` holds the number of the next sweep.
  unsigned long long sr_seed = 0;
  unsigned long long* d_sweep = nullptr;

  void* dalloc(size_t n) {
    if (n == 0) n = 256;
    void* p = nullptr;
    if (alloc) {
      p = alloc(n, alloc_ctx);
    } else if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) bytes += (int64_t)n;
    return p;
  }
  void dfree(void* p, size_t n) {
    if (!p) return;
    if (n == 0) n = 256;
    bytes -= (int64_t)n;
    if (free_)
      free_(p, alloc_ctx);
    else
      cudaFree(p);
  }
  void drop_graphs() {
    for (auto& g : graph) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
    tables_dirty = true;
  }
  void free_tables() {
    dfree(d_lat, d_lat_bytes);
    dfree(d_tiles, d_tiles_bytes);
    d_lat = nullptr;
    d_tiles = nullptr;
    d_lat_bytes = d_tiles_bytes = 0;
    ntiles = 0;
  }
};

namespace {

size_t pdf_bytes(const Lattice& L, int prec) { return (size_t)Q * (size_t)L.stride * (size_t)elem_bytes(prec); }

int cuda_fail(lbm_handle h, cudaError_t e, const char* what) {
  if (h) h->poisoned = true;
  return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, expr, what)                        \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

// After the stream is drained: did a kernel give up on a bounded wait?
int check_device_status(lbm_handle h) {
  int st = 0;
  cudaError_t e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "status word");
  if (st != 0) {
    h->poisoned = true;
    return fail(LBM_ERR_TIMEOUT, "a kernel gave up waiting for an asynchronous copy");
  }
  return LBM_OK;
}

int check_handle(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (h->poisoned) return fail(LBM_ERR_CUDA, "handle poisoned by an earlier CUDA error");
  return LBM_OK;
}

int check_lattice(lbm_handle h, int32_t lattice) {
  if (int rc = check_handle(h)) return rc;
  if (lattice < 0 || lattice >= (int32_t)h->lat.size()) return fail(LBM_ERR_ARG, "lattice index out of range");
  return LBM_OK;
}

int validate_desc(const lbm_desc* d) {
  if (!d) return fail(LBM_ERR_ARG, "null descriptor");
  if (d->nx < 2 || d->ny < 2 || d->nz < 2) return fail(LBM_ERR_ARG, "every dimension must be >= 2");
  const int64_t N = (int64_t)d->nx * d->ny * d->nz;
  if (N >= ((int64_t)1 << 31)) return fail(LBM_ERR_ARG, "lattice too large: N must be < 2^31 cells");
  if (d->precision < LBM_F64 || d->precision > LBM_F16_SHIFTED_STOCHASTIC) return fail(LBM_ERR_ARG, "bad precision");
  if (d->addressing != LBM_DIRECT && d->addressing != LBM_INDIRECT) return fail(LBM_ERR_ARG, "bad addressing");
  if (d->propagation != LBM_PULL_TWO_GRID && d->propagation != LBM_AA_INPLACE)
    return fail(LBM_ERR_ARG, "bad propagation");
  for (int a = 0; a < 3; ++a)
    if (d->periodic[a] > 1) return fail(LBM_ERR_ARG, "periodic flags must be 0 or 1");
  if (d->reserved != 0) return fail(LBM_ERR_ARG, "reserved field must be 0");
  return LBM_OK;
}

Layout current_layout(const lbm_handle h) {
  if (h->prop == LBM_PULL_TWO_GRID) return kPullForm;
  return h->phase == 0 ? kCanonical : kAAForm;
}

void* state_buffer(lbm_handle h, Lattice& L) {
  return h->prop == LBM_PULL_TWO_GRID ? L.pdf[h->phase] : L.pdf[0];
}

// RAII device scratch for one call, freed after the stream is drained.
// Device address of host memory that the GPU reads and writes in place
// (page-locked: allocated or registered with CUDA), or nullptr for ordinary
// host memory, which the calls stage through device scratch. Kernels that move
// a host array straight through the chip-to-chip link skip the copy-engine
// transfer and the scratch buffer.
void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // an unknown pointer is ordinary host memory
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

struct Scratch {
  lbm_handle h;
  void* p = nullptr;
  size_t n = 0;
  Scratch(lbm_handle h_, size_t n_) : h(h_), n(n_) { p = h->dalloc(n); }
  ~Scratch() {
    if (p) {
      cudaStreamSynchronize(h->stream);
      h->dfree(p, n);
    }
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

int create_impl(const lbm_desc* descs, int32_t count, void* stream, lbm_handle* out) {
  if (!out) return fail(LBM_ERR_ARG, "null output handle");
  *out = nullptr;
  if (!descs || count < 1 || count > 65536) return fail(LBM_ERR_ARG, "count must be in [1, 65536]");
  for (int32_t k = 0; k < count; ++k)
    if (int rc = validate_desc(descs + k)) return rc;
  for (int32_t k = 1; k < count; ++k)
    if (descs[k].precision != descs[0].precision || descs[k].propagation != descs[0].propagation)
      return fail(LBM_ERR_ARG, "all lattices of a batch must share precision and propagation");
  lbm_handle h = new lbm_lattice_s();
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    h->alloc = g_alloc;
    h->free_ = g_free;
    h->alloc_ctx = g_alloc_ctx;
  }
  h->stream = static_cast<cudaStream_t>(stream);
  h->prec = descs[0].precision;
  h->prop = descs[0].propagation;
  h->lat.resize(count);
  cudaError_t e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return fail(LBM_ERR_CUDA, std::string("stream/event creation: ") + cudaGetErrorString(e));
  }
  h->d_status = static_cast<int*>(h->dalloc(sizeof(int)));
  if (!h->d_status || cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) {
    lbm_destroy(h);
    return fail(LBM_ERR_OOM, "allocation of the status word failed");
  }
  h->d_sweep = static_cast<unsigned long long*>(h->dalloc(2 * sizeof(unsigned long long)));
  if (!h->d_sweep || cudaMemset(h->d_sweep, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    lbm_destroy(h);
    return fail(LBM_ERR_OOM, "allocation of the sweep counter failed");
  }
  for (int32_t k = 0; k < count; ++k) {
    Lattice& L = h->lat[k];
    L.status = h->d_status;
    L.desc = descs[k];
    L.N = (int64_t)L.desc.nx * L.desc.ny * L.desc.nz;
    L.flags = static_cast<uint8_t*>(h->dalloc((size_t)L.N));
    if (!L.flags) {
      lbm_destroy(h);
      return fail(LBM_ERR_OOM, "allocation of the flag field failed");
    }
  }
  *out = h;
  return LBM_OK;
}

void free_storage(lbm_handle h, Lattice& L) {
  const size_t pb = pdf_bytes(L, h->prec);
  for (auto& p : L.pdf) {
    h->dfree(p, pb);
    p = nullptr;
  }
  h->dfree(L.link, (size_t)18 * L.stride * sizeof(uint32_t));
  const int64_t chunks = ria_chunks(L.nf);
  h->dfree(L.ria_head, (size_t)chunks * 18 * sizeof(uint2));
  h->dfree(L.ria_pool, (size_t)(L.ria_pool_entries + 4) * sizeof(uint32_t));
  h->dfree(L.ria_chunk_start, (size_t)(chunks + 1) * sizeof(uint32_t));
  L.ria_head = nullptr;
  L.ria_pool = nullptr;
  L.ria_chunk_start = nullptr;
  L.ria_pool_entries = 0;
  h->dfree(L.cell_of, (size_t)L.nf * sizeof(int32_t));
  h->dfree(L.list_index, (size_t)L.N * sizeof(int32_t));
  L.link = nullptr;
  L.cell_of = L.list_index = nullptr;
}

// The run-indexed code of an indirect lattice's links (lbm_ria.cu): count the
// runs, size the pool, fill it, and check that it reproduces every link.
int build_run_index(lbm_handle h, Lattice& L) {
  const int64_t chunks = ria_chunks(L.nf);
  if (chunks == 0) return LBM_OK;
  L.ria_chunk_start = static_cast<uint32_t*>(h->dalloc((size_t)(chunks + 1) * sizeof(uint32_t)));
  L.ria_head = static_cast<uint2*>(h->dalloc((size_t)chunks * 18 * sizeof(uint2)));
  if (!L.ria_chunk_start || !L.ria_head) return fail(LBM_ERR_OOM, "allocation of the run-indexed adjacency failed");
  Scratch sc(h, 2 * sizeof(int64_t));
  if (!sc.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  const LatticeView v = L.view();
  LBM_CUDA(h, launch_ria_count(v, L.ria_chunk_start, sc.as<int64_t>(), h->stream), "run count");
  int64_t total = 0;
  LBM_CUDA(h, cudaMemcpyAsync(&total, sc.p, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream), "copy run count");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "run count sync");
  if (total <= 0 || total > 18 * L.nf) return fail(LBM_ERR_STATE, "run count of the adjacency out of range");
  L.ria_pool_entries = total;
  // 4 spare entries: a tile's pool slice is copied rounded out to 16 bytes
  L.ria_pool = static_cast<uint32_t*>(h->dalloc((size_t)(total + 4) * sizeof(uint32_t)));
  if (!L.ria_pool) return fail(LBM_ERR_OOM, "allocation of the run-indexed adjacency failed");
  LBM_CUDA(h, cudaMemsetAsync(L.ria_pool, 0, (size_t)(total + 4) * sizeof(uint32_t), h->stream), "memset pool");
  LBM_CUDA(h, launch_ria_fill(v, L.ria_chunk_start, L.ria_head, L.ria_pool, h->stream), "run fill");
  unsigned long long* d_bad = reinterpret_cast<unsigned long long*>(sc.as<int64_t>() + 1);
  LBM_CUDA(h, cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), h->stream), "memset");
  LBM_CUDA(h, launch_ria_verify(v, L.ria_head, L.ria_pool, (uint32_t)total, d_bad, h->stream), "run verify");
  unsigned long long bad = 1;
  LBM_CUDA(h, cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "copy verify");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "run verify sync");
  if (bad != 0) return fail(LBM_ERR_STATE, "run-indexed adjacency does not reproduce the link table");
  return LBM_OK;
}

// Validate the flags now on the device, build lists and allocate storage.
int finish_geometry(lbm_handle h, Lattice& L) {
  h->drop_graphs();
  L.geometry = L.init = false;
  free_storage(h, L);
  Scratch cnt(h, 10 * sizeof(unsigned long long));
  if (!cnt.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  unsigned long long* d = cnt.as<unsigned long long>();
  LBM_CUDA(h, cudaMemsetAsync(d, 0, 10 * sizeof(unsigned long long), h->stream), "memset");
  LBM_CUDA(h, launch_count_flags(L.flags, L.N, d, h->stream), "count flags");
  LBM_CUDA(h, launch_face_fluid(L.flags, L.desc.nx, L.desc.ny, L.desc.nz, d + 4, h->stream), "face check");
  unsigned long long c[10];
  LBM_CUDA(h, cudaMemcpyAsync(c, d, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "copy counts");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "geometry sync");
  if (c[3] != 0) return fail(LBM_ERR_ARG, "flags must be 0, 1 or 2");
  if (L.indirect() && c[1] != 0)
    return fail(LBM_ERR_ARG, "indirect addressing stores fluid cells only: full-way solid (flag 1) is not allowed");
  for (int a = 0; a < 3; ++a)
    if (!L.desc.periodic[a] && (c[4 + 2 * a] != 0 || c[5 + 2 * a] != 0))
      return fail(LBM_ERR_ARG, "a non-periodic dimension must be closed by solid cells on both boundary layers");
  L.nf = (int64_t)c[0];
  L.has_fullway = c[1] != 0;
  L.has_halfway = c[2] != 0;
  L.nstore = L.indirect() ? L.nf : L.N;
  L.stride = std::max<int64_t>(128, (L.nstore + 127) / 128 * 128);
  const size_t pb = pdf_bytes(L, h->prec);
  const int ngrids = h->prop == LBM_PULL_TWO_GRID ? 2 : 1;
  for (int g = 0; g < ngrids; ++g) {
    L.pdf[g] = h->dalloc(pb);
    if (!L.pdf[g]) return fail(LBM_ERR_OOM, "allocation of PDF storage failed");
    LBM_CUDA(h, cudaMemsetAsync(L.pdf[g], 0, pb, h->stream), "memset pdf");
  }
  if (L.indirect()) {
    L.list_index = static_cast<int32_t*>(h->dalloc((size_t)L.N * sizeof(int32_t)));
    L.cell_of = static_cast<int32_t*>(h->dalloc((size_t)L.nf * sizeof(int32_t)));
    if ((int64_t)Q * L.stride > (int64_t)UINT32_MAX)
      return fail(LBM_ERR_UNSUPPORTED, "fluid list too long for 32-bit link offsets (19 * stride >= 2^32)");
    L.link = static_cast<uint32_t*>(h->dalloc((size_t)18 * L.stride * sizeof(uint32_t)));
    if (!L.list_index || !L.cell_of || !L.link) return fail(LBM_ERR_OOM, "allocation of the adjacency list failed");
    LBM_CUDA(h, cudaMemsetAsync(L.link, 0, (size_t)18 * L.stride * sizeof(uint32_t), h->stream), "memset links");
    Scratch tmp(h, (size_t)scan_tmp_elems(L.N) * sizeof(int32_t));
    if (!tmp.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
    Scratch nfbuf(h, sizeof(int64_t));
    if (!nfbuf.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
    LBM_CUDA(h, launch_compact(L.flags, L.N, L.list_index, L.cell_of, tmp.as<int32_t>(), nfbuf.as<int64_t>(),
                               h->stream),
             "compaction");
    LatticeView v = L.view();
    LBM_CUDA(h, launch_links(v, L.list_index, h->prop == LBM_AA_INPLACE, L.link, h->stream), "adjacency");
    int64_t nf_check = -1;
    LBM_CUDA(h, cudaMemcpyAsync(&nf_check, nfbuf.p, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream), "copy nf");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "adjacency sync");
    if (nf_check != L.nf) return fail(LBM_ERR_STATE, "fluid compaction disagrees with the flag count");
    // every link addresses an element of the 19 direction arrays
    Scratch badbuf(h, sizeof(unsigned long long));
    if (!badbuf.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
    LBM_CUDA(h, cudaMemsetAsync(badbuf.p, 0, sizeof(unsigned long long), h->stream), "memset");
    LBM_CUDA(h, launch_links_check(L.view(), (uint64_t)Q * (uint64_t)L.stride, badbuf.as<unsigned long long>(),
                                   h->stream),
             "link check");
    unsigned long long bad = 1;
    LBM_CUDA(h, cudaMemcpyAsync(&bad, badbuf.p, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "copy link check");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "link check sync");
    if (bad != 0) return fail(LBM_ERR_STATE, "adjacency list holds offsets outside the PDF arrays");
    if (int rc = build_run_index(h, L)) return rc;
  }
  L.geometry = true;
  return LBM_OK;
}

void fill_trt(Lattice& L, double omega, double Lambda, const double F[3]) {
  L.omega = omega;
  L.Lambda = Lambda;
  L.trt.omega_p = omega;
  L.trt.omega_m = 1.0 / (Lambda / (1.0 / omega - 0.5) + 0.5);
  for (int a = 0; a < 3; ++a) L.trt.force[a] = F[a];
  for (int k = 1; k <= 9; ++k)
    L.trt.fk[k - 1] = 3.0 * weight(k) * (cx(k) * F[0] + cy(k) * F[1] + cz(k) * F[2]);
}

int ready_to_step(lbm_handle h) {
  for (size_t k = 0; k < h->lat.size(); ++k) {
    const Lattice& L = h->lat[k];
    if (!L.geometry || !L.params || !L.init)
      return fail(LBM_ERR_STATE, "lattice " + std::to_string(k) + " needs geometry, params and an initial state");
  }
  return LBM_OK;
}

// Autotuner results for the process, keyed by tune_signature().
struct TuneChoice {
  int threads, cells_per_thread, ctas_per_sm;
  bool run_indexing;
  int steps_per_pass;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;
int64_t g_tune_hits = 0;

// What the fastest launch shape depends on: the device, the storage format and
// propagation, and each lattice's size, addressing, fluid count and bounce-back kinds.
std::string tune_signature(lbm_handle h) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  std::string gpu = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? std::string(prop.name) : "gpu";
  for (char& ch : gpu)
    if (ch == ' ' || ch == '/' || ch == '\t') ch = '_';
  std::string sig = gpu + "/sm" + std::to_string(prop.multiProcessorCount) + "/p" + std::to_string(h->prec) + "/g" +
                    std::to_string(h->prop) + "/n" + std::to_string(h->lat.size());
  for (const Lattice& L : h->lat)
    sig += "/" + std::to_string(L.desc.nx) + "x" + std::to_string(L.desc.ny) + "x" + std::to_string(L.desc.nz) +
           (L.indirect() ? "i" : "d") + std::to_string(L.nf) + (L.has_fullway ? "F" : "") +
           (L.has_halfway ? "H" : "");
  return sig;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// The kernel view of lattice k with the stochastic format's stream attached.
LatticeView sweep_view(lbm_handle h, size_t k) {
  LatticeView v = h->lat[k].view();
  if (h->run_indexing && v.indirect) {
    v.ria_head = h->lat[k].ria_head;
    v.ria_pool = h->lat[k].ria_pool;
    v.ria_chunk_start = h->lat[k].ria_chunk_start;
  }
  v.sr_seed = h->sr_seed + (unsigned long long)k;
  v.sweep_ctr = h->d_sweep;
  return v;
}

// Set the number of the next sweep (device word `phase`), in stream order.
__global__ void k_set_sweep(unsigned long long* ctr, int phase, unsigned long long value) { ctr[phase] = value; }

// (Re)build the batch descriptor table and the tile work list on the device.
int build_tables(lbm_handle h) {
  if (!h->tables_dirty) return LBM_OK;
  h->free_tables();
  const size_t db = batch_lattice_bytes(h->prec);
  const int64_t tile = (int64_t)h->threads * h->cells_per_thread;
  std::vector<unsigned char> desc(db * h->lat.size());
  std::vector<BatchTile> tiles;
  for (size_t k = 0; k < h->lat.size(); ++k) {
    Lattice& L = h->lat[k];
    fill_batch_lattice(h->prec, desc.data() + k * db, sweep_view(h, k), L.pdf[0], L.pdf[1], L.trt);
    for (int64_t first = 0; first < L.nstore; first += tile)
      tiles.push_back(BatchTile{(int32_t)k, (int32_t)std::min<int64_t>(tile, L.nstore - first), first});
  }
  if (tiles.size() > (size_t)INT32_MAX) return fail(LBM_ERR_UNSUPPORTED, "too many tiles");
  h->d_lat_bytes = desc.size();
  h->d_tiles_bytes = std::max<size_t>(1, tiles.size()) * sizeof(BatchTile);
  h->d_lat = h->dalloc(h->d_lat_bytes);
  h->d_tiles = static_cast<BatchTile*>(h->dalloc(h->d_tiles_bytes));
  if (!h->d_lat || !h->d_tiles) return fail(LBM_ERR_OOM, "allocation of the batch tables failed");
  LBM_CUDA(h, cudaMemcpyAsync(h->d_lat, desc.data(), desc.size(), cudaMemcpyHostToDevice, h->stream), "copy table");
  if (!tiles.empty())
    LBM_CUDA(h, cudaMemcpyAsync(h->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice,
                                h->stream),
             "copy tiles");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "table sync");
  h->ntiles = (int)tiles.size();
  h->tables_dirty = false;
  return LBM_OK;
}

int batch_ctas(lbm_handle h, SweepKind kind) {
  if (h->ctas_per_sm <= 0) return 0;
  const int occ = batch_blocks_per_sm(h->prec, kind, h->threads);
  return sm_count() * std::min(h->ctas_per_sm, occ);
}

// Launch one time step of every lattice on stream s, at phase `phase`.
cudaError_t issue_step(lbm_handle h, int phase, cudaStream_t s) {
  if (h->batched()) {
    const SweepKind kind = h->prop == LBM_PULL_TWO_GRID ? kPull : (phase == 0 ? kAAEven : kAAOdd);
    return launch_batch_sweep(h->prec, kind, h->d_lat, h->d_tiles, h->ntiles, h->threads, batch_ctas(h, kind), phase,
                              h->d_sweep, s);
  }
  for (size_t k = 0; k < h->lat.size(); ++k) {
    Lattice& L = h->lat[k];
    const LatticeView v = sweep_view(h, k);
    cudaError_t e;
    if (h->prop == LBM_PULL_TWO_GRID)
      e = launch_sweep(v, kPull, phase, L.pdf[phase], L.pdf[phase ^ 1], L.trt, h->threads, h->cells_per_thread, s);
    else
      e = launch_sweep(v, phase == 0 ? kAAEven : kAAOdd, phase, L.pdf[0], L.pdf[0], L.trt, h->threads,
                       h->cells_per_thread, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Two time steps of a temporally blocked lattice in one launch, from buffer
// `phase` into the other one (the state then sits in buffer phase ^ 1).
cudaError_t issue_two_steps(lbm_handle h, int phase, cudaStream_t s) {
  Lattice& L = h->lat[0];
  return launch_sweep_pull2(sweep_view(h, 0), phase, L.pdf[phase], L.pdf[phase ^ 1], L.trt, s);
}

cudaError_t capture_graph(lbm_handle h, int phase, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  if (h->two_step()) {
    // kGraphSteps / 2 launches, an even number: the state returns to buffer `phase`
    for (int t = 0; t < kGraphSteps / 2 && le == cudaSuccess; ++t)
      le = issue_two_steps(h, (phase + t) & 1, h->capture_stream);
  } else {
    for (int t = 0; t < kGraphSteps && le == cudaSuccess; ++t) le = issue_step(h, (phase + t) & 1, h->capture_stream);
  }
  e = cudaStreamEndCapture(h->capture_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

int step_impl(lbm_handle h, int32_t n, bool use_graphs) {
  if (h->batched())
    if (int rc = build_tables(h)) return rc;
  int32_t done = 0;
  if (use_graphs) {
    while (n - done >= kGraphSteps) {
      cudaGraphExec_t& g = h->graph[h->phase];
      if (!g) LBM_CUDA(h, capture_graph(h, h->phase, &g), "graph capture");
      LBM_CUDA(h, cudaGraphLaunch(g, h->stream), "graph launch");
      done += kGraphSteps;   // even: phase unchanged
    }
  }
  // phase: the AA parity, or for pull the buffer that holds the state (one flip per launch)
  if (h->two_step()) {
    for (; n - done >= 2; done += 2) {
      LBM_CUDA(h, issue_two_steps(h, h->phase, h->stream), "two-step sweep launch");
      h->phase ^= 1;
    }
  }
  for (; done < n; ++done) {
    LBM_CUDA(h, issue_step(h, h->phase, h->stream), "sweep launch");
    h->phase ^= 1;
  }
  h->steps += n;
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_error.c_str(); }

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_, void* ctx) {
  if ((alloc == nullptr) != (free_ == nullptr)) return fail(LBM_ERR_ARG, "alloc and free must both be set or both NULL");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_;
  g_alloc_ctx = ctx;
  return LBM_OK;
}

int lbm_create_lattice(const lbm_desc* desc, void* cuda_stream, lbm_handle* out) {
  return create_impl(desc, 1, cuda_stream, out);
}

int lbm_create_batch(const lbm_desc* descs, int32_t count, void* cuda_stream, lbm_handle* out) {
  return create_impl(descs, count, cuda_stream, out);
}

int lbm_destroy(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  cudaStreamSynchronize(h->stream);
  h->drop_graphs();
  h->free_tables();
  for (Lattice& L : h->lat) {
    free_storage(h, L);
    h->dfree(L.flags, (size_t)L.N);
  }
  h->dfree(h->d_status, sizeof(int));
  h->dfree(h->d_sweep, 2 * sizeof(unsigned long long));
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
  return LBM_OK;
}

int lbm_set_geometry(lbm_handle h, int32_t lattice, const uint8_t* flags) {
  if (int rc = check_lattice(h, lattice)) return rc;
  if (!flags) return fail(LBM_ERR_ARG, "null flags");
  Lattice& L = h->lat[lattice];
  LBM_CUDA(h, cudaMemcpyAsync(L.flags, flags, (size_t)L.N, cudaMemcpyHostToDevice, h->stream), "copy flags");
  return finish_geometry(h, L);
}

int lbm_set_geometry_spheres(lbm_handle h, int32_t lattice, const int32_t* cxyzr, int32_t nspheres) {
  if (int rc = check_lattice(h, lattice)) return rc;
  if (nspheres < 0 || (nspheres > 0 && !cxyzr)) return fail(LBM_ERR_ARG, "bad sphere list");
  for (int32_t s = 0; s < nspheres; ++s)
    if (cxyzr[4 * s + 3] < 0) return fail(LBM_ERR_ARG, "sphere radius must be >= 0");
  Lattice& L = h->lat[lattice];
  LBM_CUDA(h, cudaMemsetAsync(L.flags, 0, (size_t)L.N, h->stream), "memset flags");
  if (nspheres > 0) {
    Scratch sph(h, (size_t)nspheres * 4 * sizeof(int32_t));
    if (!sph.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
    LBM_CUDA(h, cudaMemcpyAsync(sph.p, cxyzr, (size_t)nspheres * 4 * sizeof(int32_t), cudaMemcpyHostToDevice,
                                h->stream),
             "copy spheres");
    LBM_CUDA(h, launch_voxelize_spheres(L.desc.nx, L.desc.ny, L.desc.nz, sph.as<int32_t>(), nspheres,
                                        kSolidHalfway, L.flags, h->stream),
             "voxelize");
  }
  return finish_geometry(h, L);
}

int lbm_set_params(lbm_handle h, int32_t lattice, double omega, double Lambda, const double force[3]) {
  if (int rc = check_handle(h)) return rc;
  if (lattice < -1 || lattice >= (int32_t)h->lat.size()) return fail(LBM_ERR_ARG, "lattice index out of range");
  if (!(omega > 0.0 && omega < 2.0)) return fail(LBM_ERR_ARG, "omega must lie in (0, 2)");
  if (!(Lambda > 0.0) || !std::isfinite(Lambda)) return fail(LBM_ERR_ARG, "Lambda must be positive and finite");
  const double zero[3] = {0.0, 0.0, 0.0};
  const double* F = force ? force : zero;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(F[a])) return fail(LBM_ERR_ARG, "force must be finite");
  h->drop_graphs();
  const int32_t lo = lattice < 0 ? 0 : lattice, hi = lattice < 0 ? (int32_t)h->lat.size() : lattice + 1;
  for (int32_t k = lo; k < hi; ++k) {
    fill_trt(h->lat[k], omega, Lambda, F);
    h->lat[k].params = true;
  }
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_handle h, int32_t lattice, const double* rho, const double* u) {
  if (int rc = check_lattice(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  if (!L.geometry) return fail(LBM_ERR_STATE, "set the geometry before the initial state");
  const size_t nb = (size_t)L.N * sizeof(double);
  const double* rho_in = static_cast<const double*>(mapped_host(rho));
  const double* u_in = static_cast<const double*>(mapped_host(u));
  Scratch r(h, rho && !rho_in ? nb : 0), v(h, u && !u_in ? 3 * nb : 0);
  if ((rho && !rho_in && !r.p) || (u && !u_in && !v.p)) return fail(LBM_ERR_OOM, "scratch allocation failed");
  if (rho && !rho_in) {
    LBM_CUDA(h, cudaMemcpyAsync(r.p, rho, nb, cudaMemcpyHostToDevice, h->stream), "copy rho");
    rho_in = r.as<double>();
  }
  if (u && !u_in) {
    LBM_CUDA(h, cudaMemcpyAsync(v.p, u, 3 * nb, cudaMemcpyHostToDevice, h->stream), "copy u");
    u_in = v.as<double>();
  }
  LBM_CUDA(h, launch_from_canonical(L.view(), current_layout(h), state_buffer(h, L), nullptr, rho_in, u_in,
                                    h->stream),
           "initial state");
  k_set_sweep<<<1, 1, 0, h->stream>>>(h->d_sweep, h->phase, 0ull);
  LBM_CUDA(h, cudaGetLastError(), "sweep counter");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "init sync");
  L.init = true;
  h->steps = 0;
  return LBM_OK;
}

int lbm_write_pdfs(lbm_handle h, int32_t lattice, const double* in, size_t in_len) {
  if (int rc = check_lattice(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  if (!L.geometry) return fail(LBM_ERR_STATE, "set the geometry before writing PDFs");
  if (!in || in_len < (size_t)Q * L.N) return fail(LBM_ERR_ARG, "input must hold 19*N doubles");
  const size_t nb = (size_t)Q * L.N * sizeof(double);
  const double* direct = static_cast<const double*>(mapped_host(in));
  Scratch c(h, direct ? 0 : nb);
  if (!direct && !c.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  if (!direct) LBM_CUDA(h, cudaMemcpyAsync(c.p, in, nb, cudaMemcpyHostToDevice, h->stream), "copy pdfs");
  LBM_CUDA(h, launch_from_canonical(L.view(), current_layout(h), state_buffer(h, L), direct ? direct : c.as<double>(),
                                    nullptr, nullptr, h->stream),
           "write state");
  k_set_sweep<<<1, 1, 0, h->stream>>>(h->d_sweep, h->phase, 0ull);
  LBM_CUDA(h, cudaGetLastError(), "sweep counter");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "write sync");
  L.init = true;
  h->steps = 0;
  return LBM_OK;
}

int lbm_step(lbm_handle h, int32_t n) {
  if (int rc = check_handle(h)) return rc;
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  if (int rc = ready_to_step(h)) return rc;
  return step_impl(h, n, true);
}

int lbm_set_temporal_blocking(lbm_handle h, int32_t steps_per_pass) {
  if (int rc = check_handle(h)) return rc;
  if (steps_per_pass != 1 && steps_per_pass != 2) return fail(LBM_ERR_ARG, "steps_per_pass must be 1 or 2");
  if (steps_per_pass == 2 &&
      (h->batched() || h->prop != LBM_PULL_TWO_GRID || h->lat[0].desc.addressing != LBM_DIRECT))
    return fail(LBM_ERR_UNSUPPORTED, "temporal blocking serves a single full-array lattice with two-grid pull");
  h->drop_graphs();
  h->steps_per_pass = steps_per_pass;
  return LBM_OK;
}

int lbm_get_temporal_blocking(lbm_handle h, int32_t* steps_per_pass) {
  if (int rc = check_handle(h)) return rc;
  if (!steps_per_pass) return fail(LBM_ERR_ARG, "null output");
  *steps_per_pass = h->steps_per_pass;
  return LBM_OK;
}

int lbm_set_run_indexing(lbm_handle h, int32_t enable) {
  if (int rc = check_handle(h)) return rc;
  if (enable != 0 && enable != 1) return fail(LBM_ERR_ARG, "enable must be 0 or 1");
  h->drop_graphs();
  h->run_indexing = enable != 0;
  return LBM_OK;
}

int lbm_adjacency_bytes(lbm_handle h, int32_t lattice, int64_t out[2]) {
  if (int rc = check_lattice(h, lattice)) return rc;
  if (!out) return fail(LBM_ERR_ARG, "null output");
  const Lattice& L = h->lat[lattice];
  if (!L.geometry) return fail(LBM_ERR_STATE, "no geometry set");
  if (!L.indirect()) {
    out[0] = out[1] = 0;
    return LBM_OK;
  }
  out[0] = 18 * L.nf * (int64_t)sizeof(uint32_t);
  out[1] = ria_chunks(L.nf) * 18 * (int64_t)sizeof(uint2) + L.ria_pool_entries * (int64_t)sizeof(uint32_t);
  return LBM_OK;
}

int lbm_get_run_indexing(lbm_handle h, int32_t* enabled) {
  if (int rc = check_handle(h)) return rc;
  if (!enabled) return fail(LBM_ERR_ARG, "null output");
  *enabled = h->run_indexing ? 1 : 0;
  return LBM_OK;
}

int lbm_set_stochastic_rounding(lbm_handle h, uint64_t seed, int64_t sweep) {
  if (int rc = check_handle(h)) return rc;
  if (h->prec != LBM_F16_SHIFTED_STOCHASTIC)
    return fail(LBM_ERR_UNSUPPORTED, "stochastic rounding applies to LBM_F16_SHIFTED_STOCHASTIC storage only");
  if (sweep < 0) return fail(LBM_ERR_ARG, "the sweep number must be >= 0");
  h->drop_graphs();   // the seed is part of every captured launch
  h->sr_seed = seed;
  k_set_sweep<<<1, 1, 0, h->stream>>>(h->d_sweep, h->phase, (unsigned long long)sweep);
  LBM_CUDA(h, cudaGetLastError(), "sweep counter");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "sweep counter sync");
  return LBM_OK;
}

int lbm_synchronize(lbm_handle h) {
  if (int rc = check_handle(h)) return rc;
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  LBM_CUDA(h, cudaGetLastError(), "asynchronous error");
  return check_device_status(h);
}

int lbm_steps_done(lbm_handle h, int64_t* steps) {
  if (int rc = check_handle(h)) return rc;
  if (!steps) return fail(LBM_ERR_ARG, "null output");
  *steps = h->steps;
  return LBM_OK;
}

static int need_state(lbm_handle h, int32_t lattice) {
  if (int rc = check_lattice(h, lattice)) return rc;
  const Lattice& L = h->lat[lattice];
  if (!L.geometry || !L.init) return fail(LBM_ERR_STATE, "no state yet: set geometry and initial state first");
  return LBM_OK;
}

int lbm_read_pdfs(lbm_handle h, int32_t lattice, double* out, size_t out_len) {
  if (int rc = need_state(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  if (!out || out_len < (size_t)Q * L.N) return fail(LBM_ERR_ARG, "output must hold 19*N doubles");
  const size_t nb = (size_t)Q * L.N * sizeof(double);
  double* direct = static_cast<double*>(mapped_host(out));
  Scratch c(h, direct ? 0 : nb);
  if (!direct && !c.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  LBM_CUDA(h, launch_to_canonical(L.view(), current_layout(h), state_buffer(h, L), direct ? direct : c.as<double>(),
                                  h->stream),
           "read state");
  if (!direct) LBM_CUDA(h, cudaMemcpyAsync(out, c.p, nb, cudaMemcpyDeviceToHost, h->stream), "copy pdfs");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "read sync");
  return check_device_status(h);
}

int lbm_read_macroscopic(lbm_handle h, int32_t lattice, double* rho, double* u) {
  if (int rc = need_state(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  const size_t nb = (size_t)L.N * sizeof(double);
  double* rho_out = static_cast<double*>(mapped_host(rho));
  double* u_out = static_cast<double*>(mapped_host(u));
  Scratch r(h, rho && !rho_out ? nb : 0), v(h, u && !u_out ? 3 * nb : 0);
  if ((rho && !rho_out && !r.p) || (u && !u_out && !v.p)) return fail(LBM_ERR_OOM, "scratch allocation failed");
  LBM_CUDA(h, launch_macroscopic(L.view(), current_layout(h), state_buffer(h, L), L.trt.force,
                                 rho ? (rho_out ? rho_out : r.as<double>()) : nullptr,
                                 u ? (u_out ? u_out : v.as<double>()) : nullptr, h->stream),
           "macroscopic");
  if (rho && !rho_out) LBM_CUDA(h, cudaMemcpyAsync(rho, r.p, nb, cudaMemcpyDeviceToHost, h->stream), "copy rho");
  if (u && !u_out) LBM_CUDA(h, cudaMemcpyAsync(u, v.p, 3 * nb, cudaMemcpyDeviceToHost, h->stream), "copy u");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "macroscopic sync");
  return check_device_status(h);
}

int lbm_read_profile(lbm_handle h, int32_t lattice, int32_t axis, int32_t comp, double* out, size_t out_len) {
  if (int rc = need_state(h, lattice)) return rc;
  if (axis < 0 || axis > 2 || comp < 0 || comp > 2) return fail(LBM_ERR_ARG, "axis and comp must be 0..2");
  Lattice& L = h->lat[lattice];
  const int planes = axis == 0 ? L.desc.nx : (axis == 1 ? L.desc.ny : L.desc.nz);
  if (!out || out_len < (size_t)planes) return fail(LBM_ERR_ARG, "output must hold one value per plane");
  Scratch sc(h, (size_t)planes * (sizeof(double) + sizeof(unsigned long long)));
  if (!sc.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  double* sums = sc.as<double>();
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(sums + planes);
  LBM_CUDA(h, launch_profile(L.view(), current_layout(h), state_buffer(h, L), L.trt.force, axis, comp, sums, cnt,
                             h->stream),
           "profile");
  std::vector<double> hs(planes);
  std::vector<unsigned long long> hc(planes);
  LBM_CUDA(h, cudaMemcpyAsync(hs.data(), sums, planes * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy");
  LBM_CUDA(h, cudaMemcpyAsync(hc.data(), cnt, planes * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream),
           "copy");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "profile sync");
  for (int p = 0; p < planes; ++p) out[p] = hc[p] ? hs[p] / (double)hc[p] : 0.0;
  return check_device_status(h);
}

int lbm_read_moments(lbm_handle h, int32_t lattice, double out[4]) {
  if (int rc = need_state(h, lattice)) return rc;
  if (!out) return fail(LBM_ERR_ARG, "null output");
  Lattice& L = h->lat[lattice];
  const LatticeView v = L.view();
  const int blocks = moments_blocks(v);
  Scratch sc(h, ((size_t)blocks * 4 + 4) * sizeof(double));
  if (!sc.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  double* partials = sc.as<double>();
  double* d_out = partials + (size_t)blocks * 4;
  LBM_CUDA(h, launch_moments(v, current_layout(h), state_buffer(h, L), partials, blocks, d_out, h->stream),
           "moments");
  LBM_CUDA(h, cudaMemcpyAsync(out, d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy moments");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "moments sync");
  return check_device_status(h);
}

int lbm_read_flags(lbm_handle h, int32_t lattice, uint8_t* out, size_t out_len) {
  if (int rc = check_lattice(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  if (!L.geometry) return fail(LBM_ERR_STATE, "no geometry set");
  if (!out || out_len < (size_t)L.N) return fail(LBM_ERR_ARG, "output must hold N bytes");
  LBM_CUDA(h, cudaMemcpyAsync(out, L.flags, (size_t)L.N, cudaMemcpyDeviceToHost, h->stream), "copy flags");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "flags sync");
  return LBM_OK;
}

int lbm_fluid_count(lbm_handle h, int32_t lattice, int64_t* n_fluid) {
  if (int rc = check_lattice(h, lattice)) return rc;
  if (!n_fluid) return fail(LBM_ERR_ARG, "null output");
  if (!h->lat[lattice].geometry) return fail(LBM_ERR_STATE, "no geometry set");
  *n_fluid = h->lat[lattice].nf;
  return LBM_OK;
}

int lbm_read_adjacency(lbm_handle h, int32_t lattice, int32_t* out, size_t out_len) {
  if (int rc = check_lattice(h, lattice)) return rc;
  Lattice& L = h->lat[lattice];
  if (!L.geometry) return fail(LBM_ERR_STATE, "no geometry set");
  if (!L.indirect()) return fail(LBM_ERR_ARG, "the lattice uses direct addressing: it has no adjacency list");
  if (!out || out_len < (size_t)18 * L.nf) return fail(LBM_ERR_ARG, "output must hold 18*Nf int32");
  if (L.nf == 0) return LBM_OK;
  // the device holds element offsets; decode them back into upstream node indices
  std::vector<uint32_t> links((size_t)18 * L.nf);
  LBM_CUDA(h, cudaMemcpy2DAsync(links.data(), (size_t)L.nf * sizeof(uint32_t), L.link,
                                (size_t)L.stride * sizeof(uint32_t), (size_t)L.nf * sizeof(uint32_t), 18,
                                cudaMemcpyDeviceToHost, h->stream),
           "copy adjacency");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "adjacency sync");
  const bool aa = h->prop == LBM_AA_INPLACE;
  for (int i = 1; i < Q; ++i) {
    const uint64_t neighbour_slot = (uint64_t)(aa ? opp(i) : i);
    const uint32_t* src = links.data() + (size_t)(i - 1) * L.nf;
    int32_t* dst = out + (size_t)(i - 1) * L.nf;
    for (int64_t k = 0; k < L.nf; ++k) {
      const uint64_t off = src[k];
      const uint64_t slot = off / (uint64_t)L.stride;
      dst[k] = slot == neighbour_slot ? (int32_t)(off - slot * (uint64_t)L.stride) : -1;
    }
  }
  return LBM_OK;
}

int lbm_set_tuning(lbm_handle h, int32_t threads, int32_t cells_per_thread, int32_t ctas_per_sm) {
  if (int rc = check_handle(h)) return rc;
  if (threads >= 0 && (threads < 32 || threads > 512 || threads % 32 != 0))
    return fail(LBM_ERR_ARG, "threads must be a multiple of 32 in [32, 512]");
  if (cells_per_thread >= 0 && cells_per_thread != 1 && cells_per_thread != 2 && cells_per_thread != 4 &&
      cells_per_thread != 8)
    return fail(LBM_ERR_ARG, "cells_per_thread must be 1, 2, 4 or 8");
  if (cells_per_thread > 2 && !h->batched())
    return fail(LBM_ERR_UNSUPPORTED, "a single lattice takes 1 or 2 cells per thread");
  if (ctas_per_sm > 64) return fail(LBM_ERR_ARG, "ctas_per_sm must be <= 64");
  h->drop_graphs();
  if (threads >= 0) h->threads = threads;
  if (cells_per_thread >= 0) h->cells_per_thread = cells_per_thread;
  if (ctas_per_sm >= 0) h->ctas_per_sm = ctas_per_sm;
  return LBM_OK;
}

int lbm_get_tuning(lbm_handle h, int32_t out[3]) {
  if (int rc = check_handle(h)) return rc;
  if (!out) return fail(LBM_ERR_ARG, "null output");
  out[0] = h->threads;
  out[1] = h->cells_per_thread;
  out[2] = h->ctas_per_sm;
  return LBM_OK;
}

int lbm_autotune_cache(int64_t out[2]) {
  if (!out) return fail(LBM_ERR_ARG, "null output");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  out[0] = (int64_t)g_tune_cache.size();
  out[1] = g_tune_hits;
  return LBM_OK;
}

int lbm_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  return LBM_OK;
}

int lbm_autotune_save(const char* path) {
  if (!path) return fail(LBM_ERR_ARG, "null path");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  FILE* fp = std::fopen(path, "w");
  if (!fp) return fail(LBM_ERR_ARG, std::string("cannot write ") + path);
  std::fprintf(fp, "# lbm_gb300 autotune cache: signature threads cells_per_thread ctas_per_sm run_indexing "
                   "steps_per_pass\n");
  for (const auto& kv : g_tune_cache)
    std::fprintf(fp, "%s %d %d %d %d %d\n", kv.first.c_str(), kv.second.threads, kv.second.cells_per_thread,
                 kv.second.ctas_per_sm, kv.second.run_indexing ? 1 : 0, kv.second.steps_per_pass);
  const bool ok = std::fclose(fp) == 0;
  return ok ? LBM_OK : fail(LBM_ERR_ARG, std::string("cannot write ") + path);
}

int lbm_autotune_load(const char* path) {
  if (!path) return fail(LBM_ERR_ARG, "null path");
  FILE* fp = std::fopen(path, "r");
  if (!fp) return fail(LBM_ERR_ARG, std::string("cannot read ") + path);
  std::map<std::string, TuneChoice> read;
  char line[8192];
  int lineno = 0;
  while (std::fgets(line, sizeof(line), fp)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n') continue;
    char sig[8192];
    int t = 0, c = 0, g = 0, r = 0, spp = 0;
    if (std::sscanf(line, "%8191s %d %d %d %d %d", sig, &t, &c, &g, &r, &spp) != 6 || t < 32 || t > 512 ||
        t % 32 != 0 || (c != 1 && c != 2 && c != 4 && c != 8) || g < 0 || g > 64 || (r != 0 && r != 1) ||
        (spp != 1 && spp != 2)) {
      std::fclose(fp);
      return fail(LBM_ERR_ARG, std::string(path) + ": malformed line " + std::to_string(lineno));
    }
    read[sig] = TuneChoice{t, c, g, r == 1, spp};
  }
  std::fclose(fp);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& kv : read) g_tune_cache[kv.first] = kv.second;
  return LBM_OK;
}

int lbm_autotune(lbm_handle h, int32_t steps) {
  if (int rc = check_handle(h)) return rc;
  if (steps < 2) return fail(LBM_ERR_ARG, "steps must be >= 2");
  if (int rc = ready_to_step(h)) return rc;
  const std::string sig = tune_signature(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      ++g_tune_hits;
      h->drop_graphs();
      h->threads = it->second.threads;
      h->cells_per_thread = it->second.cells_per_thread;
      h->ctas_per_sm = it->second.ctas_per_sm;
      h->run_indexing = it->second.run_indexing;
      h->steps_per_pass = it->second.steps_per_pass;
      return LBM_OK;
    }
  }
  steps += steps & 1;   // even: the AA parity and the pull buffers come back
  // save every lattice's state so the trials leave no trace
  std::vector<void*> saved(h->lat.size(), nullptr);
  const int phase0 = h->phase;
  const int64_t steps0 = h->steps;
  unsigned long long sweep0 = 0;
  LBM_CUDA(h, cudaMemcpyAsync(&sweep0, h->d_sweep + phase0, sizeof(sweep0), cudaMemcpyDeviceToHost, h->stream),
           "save sweep counter");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "autotune sync");
  for (size_t k = 0; k < h->lat.size(); ++k) {
    Lattice& L = h->lat[k];
    saved[k] = h->dalloc(pdf_bytes(L, h->prec));
    if (!saved[k]) {
      for (size_t j = 0; j < k; ++j) h->dfree(saved[j], pdf_bytes(h->lat[j], h->prec));
      return fail(LBM_ERR_OOM, "autotune needs a copy of the state");
    }
    LBM_CUDA(h, cudaMemcpyAsync(saved[k], state_buffer(h, L), pdf_bytes(L, h->prec), cudaMemcpyDeviceToDevice,
                                h->stream),
             "save state");
  }
  struct Shape {
    int threads, cpt, ctas;
    bool ria;
    int spp;   // steps per pass
  };
  std::vector<Shape> shapes;
  if (h->batched()) {
    for (int t : {128, 256, 512})
      for (int c : {1, 2, 4, 8})
        for (int g : {0, 2, 4, 8}) shapes.push_back({t, c, g, h->run_indexing, 1});
  } else {
    const bool dense = !h->lat[0].indirect();
    for (int t : {64, 128, 192, 256, 384, 512})
      for (int c : {1, 2})
        for (int r : {1, 0})
          if ((c == 1 || dense) && (r == 1 || !dense))
            shapes.push_back({t, c, 0, dense ? h->run_indexing : r == 1, 1});
    if (dense && h->prop == LBM_PULL_TWO_GRID)   // two steps per pass: one fixed launch shape
      shapes.push_back({h->threads, h->cells_per_thread, 0, h->run_indexing, 2});
  }
  Shape best{h->threads, h->cells_per_thread, h->ctas_per_sm, h->run_indexing, h->steps_per_pass};
  float best_ms = 1e30f;
  int rc = LBM_OK;
  for (const Shape& sh : shapes) {
    h->drop_graphs();
    h->threads = sh.threads;
    h->cells_per_thread = sh.cpt;
    h->ctas_per_sm = sh.ctas;
    h->run_indexing = sh.ria;
    h->steps_per_pass = sh.spp;
    rc = step_impl(h, 2, false);   // warm-up (and table rebuild)
    if (rc == LBM_OK) {
      cudaEventRecord(h->ev0, h->stream);
      rc = step_impl(h, steps, false);
      cudaEventRecord(h->ev1, h->stream);
    }
    if (rc != LBM_OK) break;
    cudaError_t e = cudaEventSynchronize(h->ev1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (ms < best_ms) {
      best_ms = ms;
      best = sh;
    }
  }
  h->threads = best.threads;
  h->cells_per_thread = best.cpt;
  h->ctas_per_sm = best.ctas;
  h->run_indexing = best.ria;
  h->steps_per_pass = best.spp;
  h->drop_graphs();
  h->phase = phase0;
  h->steps = steps0;
  for (size_t k = 0; k < h->lat.size(); ++k) {
    Lattice& L = h->lat[k];
    LBM_CUDA(h, cudaMemcpyAsync(state_buffer(h, L), saved[k], pdf_bytes(L, h->prec), cudaMemcpyDeviceToDevice,
                                h->stream),
             "restore state");
  }
  k_set_sweep<<<1, 1, 0, h->stream>>>(h->d_sweep, phase0, sweep0);
  LBM_CUDA(h, cudaGetLastError(), "restore sweep counter");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "autotune sync");
  for (size_t k = 0; k < h->lat.size(); ++k) h->dfree(saved[k], pdf_bytes(h->lat[k], h->prec));
  if (h->poisoned) return fail(LBM_ERR_CUDA, "autotune hit a CUDA error");
  if (rc == LBM_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[sig] = TuneChoice{h->threads, h->cells_per_thread, h->ctas_per_sm, h->run_indexing,
                                   h->steps_per_pass};
  }
  return rc;
}

int lbm_memory_bytes(lbm_handle h, int64_t* bytes) {
  if (int rc = check_handle(h)) return rc;
  if (!bytes) return fail(LBM_ERR_ARG, "null output");
  *bytes = h->bytes;
  return LBM_OK;
}

int lbm_bench_copy19(const void* src, void* dst, int64_t n, int64_t stride_elems, int32_t elem_bytes,
                     void* cuda_stream) {
  if (!src || !dst || n < 0 || stride_elems < n) return fail(LBM_ERR_ARG, "bad copy-19 arguments");
  cudaError_t e = launch_copy19(src, dst, n, stride_elems, elem_bytes, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("copy-19: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_selftest_bounded_wait(lbm_handle h, int32_t polls) {
  if (int rc = check_handle(h)) return rc;
  if (polls < 1 || polls > (1 << 20)) return fail(LBM_ERR_ARG, "polls must be in [1, 2^20]");
  LBM_CUDA(h, launch_wait_selftest((uint32_t)polls, h->d_status, h->stream), "wait self-test");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "wait self-test sync");
  return check_device_status(h);
}

int lbm_bench_fma64_wave(int32_t* blocks) {
  if (!blocks) return fail(LBM_ERR_ARG, "null output");
  *blocks = fma64_wave_blocks();
  return LBM_OK;
}

int lbm_bench_fma64(double* out, int32_t blocks, int32_t iterations, void* cuda_stream) {
  if (!out || blocks < 1 || iterations < 1) return fail(LBM_ERR_ARG, "bad fma64 arguments");
  cudaError_t e = launch_fma64(out, blocks, iterations, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("fma64: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_bench_update19(void* buf, int64_t n, int64_t stride_elems, int32_t elem_bytes, void* cuda_stream) {
  if (!buf || n < 0 || stride_elems < n) return fail(LBM_ERR_ARG, "bad update-19 arguments");
  cudaError_t e = launch_update19(buf, n, stride_elems, elem_bytes, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("update-19: ") + cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lbm_read_moments_noalloc: the moments reduction with its scratch in a static
// device array instead of memory from the allocator, for callers that may not
// allocate (see the header).
namespace {

constexpr int kStaticMomentBlocks = 8192;   // covers N <= 8192 * 16384 cells
constexpr int kMaxDevices = 64;

// Block partials (4 doubles per block) followed by the 4 final sums. Every
// slot a call reads is written earlier in the same call, so nothing needs
// clearing between calls.
static __device__ __align__(256) double g_moment_scratch[kStaticMomentBlocks * 4 + 4];

std::mutex g_static_mu;
double* g_static_scratch[kMaxDevices] = {};

// Device address of g_moment_scratch on `dev`, looked up once per device with
// that device current. The host-side name is only a stand-in for the symbol.
int static_scratch(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_scratch[dev]) {
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_moment_scratch);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_static_scratch[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_read_moments_noalloc(lbm_handle h, int32_t lattice, double out[4]) {
  if (int rc = need_state(h, lattice)) return rc;
  if (!out) return fail(LBM_ERR_ARG, "null output");
  Lattice& L = h->lat[lattice];
  const LatticeView v = L.view();
  const int blocks = moments_blocks(v);
  if (blocks > kStaticMomentBlocks)
    return fail(LBM_ERR_ARG, "lattice too large for the static scratch of lbm_read_moments_noalloc: "
                             "N must be <= 134217728 cells");
  void* state = state_buffer(h, L);
  cudaPointerAttributes attr{};
  LBM_CUDA(h, cudaPointerGetAttributes(&attr, state), "device of the lattice");
  double* scratch = nullptr;
  if (int rc = static_scratch(attr.device, &scratch)) return rc;
  double* d_out = scratch + (size_t)kStaticMomentBlocks * 4;
  LBM_CUDA(h, launch_moments(v, current_layout(h), state, scratch, blocks, d_out, h->stream), "moments");
  LBM_CUDA(h, cudaMemcpyAsync(out, d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy moments");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "moments sync");
  // Report a bounded wait that gave up in an earlier sweep, as lbm_read_moments does.
  return check_device_status(h);
}

// C ABI of libsph.so: handle lifetime, parameter checks, per-tank constants,
// the host-driven and graph-driven advection loops, state import/export.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <initializer_list>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <sys/types.h>

#include "sph.h"
#include "sph_handle.h"
#include "sph_kernels.h"

const char* sph_noalloc_last_error();   // message of the last failed handle-less call (sph_noalloc.cu)

using sph::Buffers;
using sph::Ctrl;
using sph::Global;
using sph::Inst;


namespace {

constexpr int kQuantBits = 22;

int make_dir(const std::string& dir) { return mkdir(dir.c_str(), 0755); }

int fail(sph_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(sph_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? SPH_E_OOM : SPH_E_CUDA, m);
}

#define CK(h, call)                                            \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);   \
  } while (0)

template <typename T>
int dalloc(sph_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
  h->allocs.push_back((void*)*p);
  h->device_bytes += (int64_t)(sizeof(T) * count);
  return SPH_OK;
}

#define DALLOC(h, p, n)                    \
  do {                                     \
    int r_ = dalloc((h), &(p), (n));       \
    if (r_ != SPH_OK) return r_;           \
  } while (0)

int bitlength(long long v) {
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Wendland C2 in double (host): W(r) = alpha (1 - q/2)^4 (1 + 2q), q = r/h < 2.
double wendland_alpha(double h, int dim) {
  const double pi = 3.14159265358979323846;
  return dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
}

double wendland_W(double r, double h, int dim) {
  double q = r / h;
  if (q >= 2.0) return 0.0;
  double t = 1.0 - 0.5 * q;
  return wendland_alpha(h, dim) * t * t * t * t * (1.0 + 2.0 * q);
}

// sum_k W(|k| dp) over the square / cubic lattice, self included.
double lattice_sum(double dp, double h, int dim) {
  int kmax = (int)std::ceil(2.0 * h / dp) + 1;
  double s = 0.0;
  for (int kz = (dim == 3 ? -kmax : 0); kz <= (dim == 3 ? kmax : 0); ++kz)
    for (int ky = -kmax; ky <= kmax; ++ky)
      for (int kx = -kmax; kx <= kmax; ++kx) {
        double r = dp * std::sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
        s += wendland_W(r, h, dim);
      }
  return s;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_params(const sph_params* p, std::string* why) {
  auto bad = [&](const char* m) {
    if (why) *why = m;
    return SPH_E_INVALID;
  };
  if (!p) return bad("params is NULL");
  if (p->dim != 2 && p->dim != 3) return bad("dim must be 2 or 3");
  if (!finite_pos(p->h)) return bad("h must be positive");
  if (!finite_pos(p->dp)) return bad("dp must be positive");
  if (!finite_pos(p->rho0)) return bad("rho0 must be positive");
  if (!finite_pos(p->c0)) return bad("c0 must be positive");
  if (!finite_pos(p->cfl_ad) || !finite_pos(p->cfl_ac)) return bad("CFL numbers must be positive");
  if (!(std::isfinite(p->u_ref) && p->u_ref >= 0.0)) return bad("u_ref must be >= 0");
  if (!(std::isfinite(p->nu) && p->nu >= 0.0)) return bad("nu must be >= 0");
  if (p->u_ref == 0.0 && !(p->nu > 0.0)) return bad("u_ref = 0 needs nu > 0 to bound Dt_ad");
  if (p->capacity < 0 || p->capacity > 65535) return bad("capacity must be in [0, 65535]");
  if (p->free_surface != 0 && p->free_surface != 1) return bad("free_surface must be 0 or 1");
  if (!(std::isfinite(p->p_transport) && p->p_transport >= 0.0)) return bad("p_transport must be >= 0");
  if (p->max_substeps < 0) return bad("max_substeps must be >= 0");
  if (p->flags & SPH_FLAG_HALF_PAIR) {
    if (p->flags & SPH_FLAG_FROZEN_GEOMETRY) return bad("the half-pair evaluation recomputes the pair geometry");
    if (p->p_transport > 0.0) return bad("the half-pair evaluation has no transport velocity");
    if (p->capacity > 252) return bad("the half-pair evaluation needs capacity <= 252");
  }
  if (p->p_transport > 0.0 && (p->flags & SPH_FLAG_FROZEN_GEOMETRY))
    return bad("the transport velocity needs the recomputed pair geometry (no SPH_FLAG_FROZEN_GEOMETRY)");
  double period = 0.0;
  for (int a = 0; a < p->dim; ++a) {
    if (!std::isfinite(p->gravity[a])) return bad("gravity must be finite");
    if (!(std::isfinite(p->lo[a]) && std::isfinite(p->hi[a]) && p->hi[a] > p->lo[a]))
      return bad("need lo < hi on every axis");
    if (p->periodic[a] != 0 && p->periodic[a] != 1) return bad("periodic must be 0 or 1");
    if (p->periodic[a]) {
      double L = p->hi[a] - p->lo[a];
      if (period == 0.0) period = L;
      else if (L != period) return bad("all periodic axes must share one period");
      if (std::floor(L / (2.0 * p->h)) < 3.0) return bad("a periodic axis needs at least 3 cells");
    }
  }
  double cell = period > 0.0 ? period / std::floor(period / (2.0 * p->h)) : 2.0 * p->h;
  for (int a = 0; a < p->dim; ++a) {
    double nc = p->periodic[a] ? std::floor(period / (2.0 * p->h)) : std::ceil((p->hi[a] - p->lo[a]) / cell);
    if (nc > 32768.0) return bad("more than 32768 cells on an axis");
  }
  return SPH_OK;
}

// Per-tank constants, following the position contract in sph.h.
Inst make_inst(const sph_params& p) {
  Inst I;
  std::memset(&I, 0, sizeof(I));
  const int d = p.dim;
  double period = 0.0;
  for (int a = 0; a < d; ++a)
    if (p.periodic[a]) period = p.hi[a] - p.lo[a];
  double cell = period > 0.0 ? period / std::floor(period / (2.0 * p.h)) : 2.0 * p.h;
  int ncell[3] = {1, 1, 1};
  int nmax = 1;
  for (int a = 0; a < d; ++a) {
    if (p.periodic[a]) ncell[a] = (int)std::floor(period / (2.0 * p.h));
    else ncell[a] = std::max(1, (int)std::ceil((p.hi[a] - p.lo[a]) / cell));
    nmax = std::max(nmax, ncell[a]);
  }
  int bits = std::min(kQuantBits, 31 - bitlength(nmax));
  double dq = cell / (double)(1u << bits);
  double x = 2.0 * p.h / dq;
  long long R2 = (long long)std::ceil(x * x);
  const double alpha = wendland_alpha(p.h, d);
  const double sigma0 = lattice_sum(p.dp, p.h, d);
  const double sig = alpha - sigma0;        // W(0) - sumW0
  I.h = (float)p.h;
  I.inv_h = (float)(1.0 / p.h);
  I.four_h2 = (float)(4.0 * p.h * p.h);
  I.dq = (float)dq;
  I.inv_dq = (float)(1.0 / dq);
  I.c0 = (float)p.c0;
  I.c0sq = (float)(p.c0 * p.c0);
  I.rho0 = (float)p.rho0;
  I.w_a = (float)alpha;
  I.dwr_a = (float)(-5.0 * alpha / (p.h * p.h));
  I.sig_hi = (float)sig;
  I.sig_lo = (float)(sig - (double)I.sig_hi);
  I.rho0_over_sigma0 = (float)(p.rho0 / sigma0);
  I.kc = sph::kLimiter / I.c0;                   // FP32 operations, as on the device
  I.qc0 = 0.25f * I.c0;
  I.hc0sq = 0.5f * I.c0sq;
  I.inv_c0sq = 1.0f / I.c0sq;
  for (int a = 0; a < 3; ++a) I.g[a] = a < d ? (float)p.gravity[a] : 0.0f;
  I.eta = (float)(p.rho0 * p.nu);
  I.mass = 0.0f;
  I.p_tv = (float)p.p_transport;
  I.max_sub = p.max_substeps > 0 ? p.max_substeps : sph::kMaxSubstepsPerStep;
  for (int a = 0; a < 3; ++a) {
    I.ncell[a] = ncell[a];
    I.scell[a] = a < d ? 2 * ncell[a] : 1;
    I.period[a] = (a < d && p.periodic[a]) ? (ncell[a] << bits) : 0;
    I.lo[a] = a < d ? p.lo[a] : 0.0;
  }
  I.bits = bits;
  I.sbits = bits - 1;
  I.free_surface = p.free_surface;
  I.R2 = R2;
  I.h_d = p.h;
  I.c0_d = p.c0;
  I.u_ref = p.u_ref;
  I.nu = p.nu;
  I.cfl_ad = p.cfl_ad;
  I.cfl_ac = p.cfl_ac;
  I.dq_d = dq;
  I.rho0_d = p.rho0;
  return I;
}

// Memory the current device addresses directly: its own device memory or managed memory.
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.device == cur;
}

// Device memory of a GPU other than the current one. The kernels run on the current
// device, so the entry points reject such arrays instead of dereferencing them.
bool foreign_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int cur = -1;
  if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.device != cur;
}

bool any_foreign(std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs)
    if (foreign_device_ptr(p)) return true;
  return false;
}

int status_code(const Global& g) {
  if (g.err & sph::ERR_BOUNDS) return SPH_E_BOUNDS;
  if (g.err & sph::ERR_DOMAIN) return SPH_E_DOMAIN;
  if (g.err & sph::ERR_CAPACITY) return SPH_E_CAPACITY;
  if (g.err & (sph::ERR_NAN | sph::ERR_DT)) return SPH_E_UNSTABLE;
  if (g.err & sph::ERR_TIMEOUT) return SPH_E_TIMEOUT;
  return SPH_OK;
}

// Synchronise `s`, read the device status and turn error bits into a code.
int sync_status(sph_handle* h, cudaStream_t s) {
  CK(h, cudaMemcpyAsync(h->hglob, h->b.glob, sizeof(Global), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  int code = status_code(*h->hglob);
  if (code != SPH_OK) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "device error bits 0x%x (first at slot %lld)", h->hglob->err,
                  (long long)h->hglob->bad_index);
    h->err = buf;
  }
  return code;
}

// The row pieces of the row-task form, built with the cells when a relaxation uses it
// (otherwise at that relaxation's first launch after the build).
void enqueue_row_tasks(sph_handle* h, cudaStream_t s, int64_t* n) {
  const sph::LaunchCfg& c = h->b.cfg;
  if (h->b.row_task && !h->b.geo && (sph::row_form(c.pr_block) || sph::row_form(c.dr_block))) {
    sph::launch_row_tasks(h->b, s, n);
    h->rows_valid = true;
  }
}

void enqueue_build(sph_handle* h, cudaStream_t s, int64_t* n) {
  sph::launch_hash(h->b, s, n);
  sph::launch_fluid_offsets(h->b, s, n);
  sph::launch_sort_fluid(h->b, s, n);
  sph::launch_neighbours(h->b, s, n);
  enqueue_row_tasks(h, s, n);
  sph::launch_reverse_slots(h->b, s, n);     // half-pair evaluation only (b.hrev set)
  sph_fsi_after_build(h, s, n);              // attached solid only
}

bool debug_bounds(const sph_handle* h) { return (h->flags & SPH_FLAG_DEBUG_BOUNDS) != 0; }

// SPH_FLAG_DEBUG_BOUNDS: check the cell offsets and the neighbour table, synchronously,
// before anything reads them; SPH_OK when the flag is off.
int debug_check(sph_handle* h, cudaStream_t s) {
  if (!debug_bounds(h)) return SPH_OK;
  sph::launch_check_offsets(h->b, s, &h->launches);
  sph::launch_check_table(h->b, s, &h->launches);
  CK(h, cudaGetLastError());
  return sync_status(h, s);
}

// Configuration update. With SPH_FLAG_DEBUG_BOUNDS the offsets are checked after the scan
// and before the scatter and the neighbour search read them, and the new table after it is
// written; otherwise the four stages are only enqueued.
int run_build(sph_handle* h, cudaStream_t s) {
  if (!debug_bounds(h)) {
    enqueue_build(h, s, &h->launches);
    CK(h, cudaGetLastError());
    return SPH_OK;
  }
  sph::launch_hash(h->b, s, &h->launches);
  sph::launch_fluid_offsets(h->b, s, &h->launches);
  sph::launch_check_offsets(h->b, s, &h->launches);
  CK(h, cudaGetLastError());
  int r = sync_status(h, s);
  if (r != SPH_OK) return r;
  sph::launch_sort_fluid(h->b, s, &h->launches);
  sph::launch_neighbours(h->b, s, &h->launches);
  sph::launch_check_table(h->b, s, &h->launches);
  enqueue_row_tasks(h, s, &h->launches);
  CK(h, cudaGetLastError());
  int rt = sync_status(h, s);              // the reverse map reads the table: check it first
  if (rt != SPH_OK) return rt;
  sph::launch_reverse_slots(h->b, s, &h->launches);
  sph_fsi_after_build(h, s, &h->launches);
  CK(h, cudaGetLastError());
  return sync_status(h, s);
}

void enqueue_advection(sph_handle* h, cudaStream_t s, int64_t* n) {
  sph::launch_dt_advection(h->b, s, n);
  sph::launch_density(h->b, s, n);
  sph::launch_viscous(h->b, s, n);
  sph::launch_pair_geometry(h->b, s, n);     // frozen-geometry reading only (b.geo set)
}

void enqueue_substep(sph_handle* h, cudaStream_t s, bool use_cond, int64_t* n) {
  sph::launch_dt_acoustic(h->b, s, h->cond, use_cond, n);
  if (h->timing && !use_cond) cudaEventRecord(h->ev[0], s);
  if (h->b.hrev) sph::launch_half_pair(h->b, true, s, n);
  else sph::launch_pressure_relaxation(h->b, s, n);
  sph_fsi_after_pressure(h, s, n);
  if (h->timing && !use_cond) cudaEventRecord(h->ev[1], s);
  if (h->b.hrev) sph::launch_half_pair(h->b, false, s, n);
  else sph::launch_density_relaxation(h->b, s, n);
  sph_fsi_after_density(h, s, n);
  if (h->timing && !use_cond) cudaEventRecord(h->ev[2], s);
}

int build_graph(sph_handle* h) {
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t g = nullptr;
  CK(h, cudaGraphCreate(&g, 0));
  CK(h, cudaGraphConditionalHandleCreate(&h->cond, g, 1, cudaGraphCondAssignDefault));
  int64_t fixed = 0, body_n = 0;
  CK(h, cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enqueue_build(h, cs, &fixed);
  enqueue_advection(h, cs, &fixed);
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(h, cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(h, cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(h, cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(h, cudaStreamEndCapture(cs, &g));
  CK(h, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enqueue_substep(h, cs, true, &body_n);
  CK(h, cudaStreamEndCapture(cs, &body));
  CK(h, cudaGraphInstantiate(&h->gexec, g, 0));
  h->graph = g;
  h->graph_fixed = fixed;
  h->graph_body = body_n;
  return SPH_OK;
}

int ensure_stage(sph_handle* h, size_t elems) {
  if (h->stage_elems >= elems) return SPH_OK;
  if (h->stage) {
    cudaFree(h->stage);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)h->stage), h->allocs.end());
    h->device_bytes -= (int64_t)(h->stage_elems * sizeof(double));
    h->stage = nullptr;
  }
  DALLOC(h, h->stage, elems);
  h->stage_elems = elems;
  return SPH_OK;
}

constexpr int kUploadChunks = 8;              // host state upload: chunks (and events - 1)
constexpr int64_t kUploadChunkMin = 1 << 18;  // particles below which one copy is enough

// Bring caller arrays onto the device: device pointers are used as they are,
// host arrays go through the staging buffer at offset `off`.
const double* device_view(sph_handle* h, const double* p, size_t elems, size_t off, cudaStream_t s,
                          cudaError_t* e) {
  *e = cudaSuccess;
  if (!p || is_device_ptr(p)) return p;
  *e = cudaMemcpyAsync(h->stage + off, p, sizeof(double) * elems, cudaMemcpyHostToDevice, s);
  return h->stage + off;
}

// ---------------------------------------------------------------- autotuner ----------
// Launch variants of the two acoustic-substep kernels: threads per particle x block size.
// The choice is cached per (GPU, dimension, particle-count bucket, batched or not) in a
// small JSON file: $SPH_AUTOTUNE_CACHE, else $HOME/.cache/sph_gb300_autotune.json.
const int kTppChoices[3] = {1, 2, 4};
const int kBlockChoices[3] = {128, 256, 512};
// per kernel: the 3 x 3 (threads per particle, block) variants, then the row-task form
constexpr int kAutotuneVariants = 10;

std::string autotune_path() {
  const char* env = std::getenv("SPH_AUTOTUNE_CACHE");
  if (env && *env) return env;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/sph_gb300_autotune.json";
}

std::string autotune_key(const sph_handle* h) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) cudaGetLastError();
  int bucket = 0;
  for (int64_t v = std::max<int64_t>(h->b.n, 1); v > 1; v >>= 1) ++bucket;
  std::ostringstream k;
  k << prop.name << "|d" << h->b.dim << "|n2^" << bucket << "|" << (h->b.n_inst > 1 ? "batched" : "single");
  return k.str();
}

// The cache is a flat JSON object {"key": "pr_tpp,pr_block,dr_tpp,dr_block", ...}.
std::map<std::string, std::string> read_autotune_cache() {
  std::map<std::string, std::string> m;
  std::ifstream f(autotune_path());
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  size_t p = 0;
  while (true) {
    size_t a = t.find('"', p);
    if (a == std::string::npos) break;
    size_t b = t.find('"', a + 1);
    if (b == std::string::npos) break;
    size_t c = t.find('"', b + 1);
    if (c == std::string::npos) break;
    size_t d = t.find('"', c + 1);
    if (d == std::string::npos) break;
    m[t.substr(a + 1, b - a - 1)] = t.substr(c + 1, d - c - 1);
    p = d + 1;
  }
  return m;
}

void write_autotune_cache(const std::map<std::string, std::string>& m) {
  const std::string path = autotune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)          // mkdir -p, component by component
      if (i == dir.size() || dir[i] == '/') (void)make_dir(dir.substr(0, i));
  }
  std::ofstream f(path + ".tmp");
  if (!f) return;
  f << "{\n";
  size_t k = 0;
  for (const auto& kv : m) f << "  \"" << kv.first << "\": \"" << kv.second << "\"" << (++k < m.size() ? ",\n" : "\n");
  f << "}\n";
  f.close();
  std::rename((path + ".tmp").c_str(), path.c_str());
}

// "pr_tpp,pr_block,dr_tpp,dr_block"; the row-task form (block kRowBlock, one thread per
// particle) only for a handle of one tank.
bool parse_cfg(const std::string& v, sph::LaunchCfg* c, bool single) {
  int a[4];
  if (std::sscanf(v.c_str(), "%d,%d,%d,%d", &a[0], &a[1], &a[2], &a[3]) != 4) return false;
  auto ok_t = [](int t) { return t == 1 || t == 2 || t == 4; };
  auto ok_b = [](int b) { return b == 128 || b == 256 || b == 512; };
  auto ok = [&](int t, int b) { return ok_t(t) && (ok_b(b) || (single && t == 1 && sph::row_form(b))); };
  if (!ok(a[0], a[1]) || !ok(a[2], a[3])) return false;
  c->pr_tpp = a[0];
  c->pr_block = a[1];
  c->dr_tpp = a[2];
  c->dr_block = a[3];
  return true;
}

std::string format_cfg(const sph::LaunchCfg& c) {
  std::ostringstream o;
  o << c.pr_tpp << "," << c.pr_block << "," << c.dr_tpp << "," << c.dr_block;
  return o.str();
}

void drop_graph(sph_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
}

}  // namespace

int sph_sync_status(sph_handle* h, cudaStream_t s) { return sync_status(h, s); }
void sph_drop_graph(sph_handle* h) { drop_graph(h); }
int sph_debug_check(sph_handle* h, cudaStream_t s) { return debug_check(h, s); }

extern "C" {

int sph_params_check(const sph_params* p) { return check_params(p, nullptr); }

const char* sph_last_error(const sph_handle* h) { return h ? h->err.c_str() : sph_noalloc_last_error(); }

void sph_destroy(sph_handle* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->up_stream) cudaStreamDestroy(h->up_stream);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->up_ev)
    if (e) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hglob) cudaFreeHost(h->hglob);
  delete h;
}

int sph_create(const sph_params* params, int32_t n_instances, const int64_t* fluid_offsets,
               const int64_t* wall_offsets, int64_t n_fluid, const double* pos, const double* vel,
               const double* rho, const double* mass, int64_t n_wall, const double* wall_pos,
               const double* wall_normal, const double* wall_vol, void* stream, sph_handle** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (!params || n_instances < 1 || n_fluid < 0 || n_wall < 0) return SPH_E_INVALID;
  if (n_fluid > 0 && (!pos || !vel || !rho || !mass)) return SPH_E_INVALID;
  if (n_wall > 0 && (!wall_pos || !wall_normal || !wall_vol)) return SPH_E_INVALID;
  if (n_instances > 1 && (!fluid_offsets || !wall_offsets)) return SPH_E_INVALID;
  if (n_fluid >= (1ll << 31) || n_wall >= (1ll << 31)) return SPH_E_INVALID;
  if (any_foreign({pos, vel, rho, mass, wall_pos, wall_normal, wall_vol})) return SPH_E_INVALID;
  for (int k = 0; k < n_instances; ++k) {
    if (check_params(&params[k], nullptr) != SPH_OK) return SPH_E_INVALID;
    if (params[k].dim != params[0].dim) return SPH_E_INVALID;
  }
  std::vector<int64_t> fo(n_instances + 1), wo(n_instances + 1);
  if (n_instances == 1) {
    fo[0] = 0; fo[1] = n_fluid; wo[0] = 0; wo[1] = n_wall;
  } else {
    for (int k = 0; k <= n_instances; ++k) {
      fo[k] = fluid_offsets[k];
      wo[k] = wall_offsets[k];
    }
  }
  if (fo[0] != 0 || fo[n_instances] != n_fluid || wo[0] != 0 || wo[n_instances] != n_wall)
    return SPH_E_INVALID;
  for (int k = 0; k < n_instances; ++k)
    if (fo[k + 1] < fo[k] || wo[k + 1] < wo[k]) return SPH_E_INVALID;

  sph_handle* h = new sph_handle();
  *out = h;
  cudaStream_t s = (cudaStream_t)stream;
  const int dim = params[0].dim;
  h->params.assign(params, params + n_instances);
  h->flags = params[0].flags;
  Buffers& b = h->b;
  b.n = n_fluid;
  b.nw = n_wall;
  b.n_inst = n_instances;
  b.dim = dim;
  b.cap = params[0].capacity > 0 ? params[0].capacity : (dim == 2 ? 48 : 128);
  b.cap = (b.cap + 3) & ~3;                  // whole quads of neighbour slots
  int64_t n_cells = 0;
  bool any_visc = false;
  for (int k = 0; k < n_instances; ++k) {
    Inst I = make_inst(params[k]);
    I.cell_base = n_cells;
    long long nc = 1;
    for (int a = 0; a < dim; ++a) nc *= I.scell[a];
    n_cells += nc;
    I.fluid_begin = fo[k];
    I.fluid_end = fo[k + 1];
    I.wall_begin = wo[k];
    I.wall_end = wo[k + 1];
    if (params[k].nu > 0.0) any_visc = true;
    for (int a = 0; a < dim; ++a)
      if (params[k].periodic[a]) b.any_periodic = true;
    if (params[k].p_transport > 0.0) b.any_transport = true;
    h->hinst.push_back(I);
  }
  if (n_cells >= (1ll << 32) - 1) return fail(h, SPH_E_INVALID, "too many cells");
  b.n_cells = n_cells;

  // masses: one value per tank when uniform, else a per-particle array
  std::vector<double> hm(n_fluid);
  if (n_fluid) {
    cudaError_t e = cudaMemcpy(hm.data(), mass, sizeof(double) * n_fluid, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy masses");
  }
  bool uniform = true;
  for (int k = 0; k < n_instances; ++k) {
    for (int64_t i = fo[k]; i < fo[k + 1]; ++i)
      if (hm[i] != hm[fo[k]]) uniform = false;
    if (fo[k + 1] > fo[k]) h->hinst[k].mass = (float)hm[fo[k]];
  }

  const int64_t nmax = std::max<int64_t>(n_fluid, n_wall);
  DALLOC(h, b.inst, n_instances);
  DALLOC(h, b.ctrl, n_instances);
  DALLOC(h, b.glob, 1);
  DALLOC(h, b.pbar, 1);
  DALLOC(h, b.PS, n_fluid);
  DALLOC(h, b.VS, n_fluid);
  DALLOC(h, b.PH, nmax);
  DALLOC(h, b.VH, nmax);
  DALLOC(h, b.id, n_fluid);
  DALLOC(h, b.cell, nmax);
  DALLOC(h, b.rank, nmax);
  DALLOC(h, b.key, nmax);
  DALLOC(h, b.src, nmax);
  DALLOC(h, b.count, n_cells);
  DALLOC(h, b.fstart, n_cells + 1);
  DALLOC(h, b.wstart, n_cells + 1);
  DALLOC(h, b.wnear, n_cells);
  DALLOC(h, b.scan_tmp, sph::scan_tmp_elems(n_cells));
  if (n_instances == 1 && n_fluid > 0) {      // row pieces of the row-task form
    const Inst& I0 = h->hinst[0];
    b.n_rows = (int64_t)I0.scell[1] * I0.scell[2];
    b.row_task_cap = (n_fluid + 31) / 32 + b.n_rows;   // sum over rows of ceil(len / 32)
    DALLOC(h, b.row_task, (size_t)b.row_task_cap);
    DALLOC(h, b.row_cnt, (size_t)b.n_rows);
    DALLOC(h, b.row_off, (size_t)b.n_rows + 1);
    DALLOC(h, b.row_tmp, sph::scan_tmp_elems(b.n_rows));
  }
  b.rows_valid = &h->rows_valid;
  {
    int dev = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&b.n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  DALLOC(h, b.WP, n_wall);
  DALLOC(h, b.WN, n_wall);
  DALLOC(h, b.wid, n_wall);
  DALLOC(h, b.nbr, (size_t)n_fluid * b.cap);
  DALLOC(h, b.nbc, n_fluid);
  if (!uniform) {
    DALLOC(h, b.mass, n_fluid);
    DALLOC(h, b.mass_tmp, n_fluid);
    std::vector<float> fm(hm.begin(), hm.end());
    CK(h, cudaMemcpy(b.mass, fm.data(), sizeof(float) * n_fluid, cudaMemcpyHostToDevice));
  }
  if (any_visc) {
    DALLOC(h, b.acc_prior, n_fluid);
    CK(h, cudaMemset(b.acc_prior, 0, sizeof(float4) * std::max<int64_t>(n_fluid, 1)));
  }
  if (h->flags & SPH_FLAG_FROZEN_GEOMETRY) DALLOC(h, b.geo, (size_t)n_fluid * b.cap);
  if (h->flags & SPH_FLAG_HALF_PAIR) {
    DALLOC(h, b.hshare, (size_t)n_fluid * b.cap);
    DALLOC(h, b.hpart, n_fluid);
    DALLOC(h, b.hrev, (size_t)n_fluid * b.cap);
  }
  if (h->flags & SPH_FLAG_KEEP_ACC) {
    DALLOC(h, b.acc_keep, n_fluid);
    CK(h, cudaMemset(b.acc_keep, 0, sizeof(float4) * std::max<int64_t>(n_fluid, 1)));
  }
  if (n_instances > 1) {
    std::vector<int> io(n_fluid), wio(n_wall);
    for (int k = 0; k < n_instances; ++k) {
      for (int64_t i = fo[k]; i < fo[k + 1]; ++i) io[i] = k;
      for (int64_t i = wo[k]; i < wo[k + 1]; ++i) wio[i] = k;
    }
    int *dio = nullptr, *dwio = nullptr;
    DALLOC(h, dio, n_fluid);
    DALLOC(h, dwio, n_wall);
    if (n_fluid) CK(h, cudaMemcpy(dio, io.data(), sizeof(int) * n_fluid, cudaMemcpyHostToDevice));
    if (n_wall) CK(h, cudaMemcpy(dwio, wio.data(), sizeof(int) * n_wall, cudaMemcpyHostToDevice));
    b.inst_of = dio;
    b.winst_of = dwio;
  }
  DALLOC(h, h->diag_scratch, sph::diag_scratch_elems(b));
  DALLOC(h, h->diag_out, (size_t)n_instances * sph::kDiagFields);
  CK(h, cudaMallocHost((void**)&h->hglob, sizeof(Global)));
  {
    int r = ensure_stage(h, std::max<size_t>((size_t)n_fluid * (2 * dim + 2), (size_t)n_wall * (2 * dim + 1)));
    if (r != SPH_OK) return r;
  }
  CK(h, cudaMemcpy(b.inst, h->hinst.data(), sizeof(Inst) * n_instances, cudaMemcpyHostToDevice));
  b.inst0 = h->hinst[0];
  std::vector<Ctrl> hc(n_instances);
  std::memset(hc.data(), 0, sizeof(Ctrl) * n_instances);
  CK(h, cudaMemcpy(b.ctrl, hc.data(), sizeof(Ctrl) * n_instances, cudaMemcpyHostToDevice));
  CK(h, cudaMemset(b.glob, 0, sizeof(Global)));
  CK(h, cudaMemset(b.pbar, 0, sizeof(sph::GridBarrier)));
  for (auto& e : h->ev) CK(h, cudaEventCreate(&e));

  // walls: import and sort into cells once
  if (n_wall) {
    cudaError_t e1, e2, e3;
    const double* wp = device_view(h, wall_pos, (size_t)n_wall * dim, 0, s, &e1);
    const double* wn = device_view(h, wall_normal, (size_t)n_wall * dim, (size_t)n_wall * dim, s, &e2);
    const double* wv = device_view(h, wall_vol, (size_t)n_wall, (size_t)n_wall * dim * 2, s, &e3);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
      return cuda_fail(h, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "copy walls");
    sph::launch_import_walls(b, wp, wn, wv, s);
    CK(h, cudaStreamSynchronize(s));
  }
  sph::sort_walls(b, b.PH, b.VH, b.wid, s);
  sph::flag_near_wall_cells(b, reinterpret_cast<uint8_t*>(b.count), s);   // count: scratch here
  {
    const auto cache = read_autotune_cache();
    const auto it = cache.find(autotune_key(h));
    if (it != cache.end()) parse_cfg(it->second, &b.cfg, n_instances == 1);
  }
  CK(h, cudaGetLastError());
  int r = sph_set_state(h, pos, vel, rho, nullptr, 0.0, stream);
  if (r != SPH_OK) return r;
  return sync_status(h, s);
}

int sph_get_info(const sph_handle* h, sph_info* out) {
  if (!h || !out) return SPH_E_INVALID;
  const Inst& I = h->hinst[0];
  out->dim = h->b.dim;
  out->n_instances = h->b.n_inst;
  out->capacity = h->b.cap;
  out->bits = I.bits;
  out->n_fluid = h->b.n;
  out->n_wall = h->b.nw;
  out->n_cells = h->b.n_cells;
  out->cell = I.dq_d * (double)(1u << I.bits);
  out->dq = I.dq_d;
  out->sigma0 = lattice_sum(h->params[0].dp, h->params[0].h, h->b.dim);
  out->R2 = I.R2;
  out->device_bytes = h->device_bytes;
  return SPH_OK;
}

int sph_set_state(sph_handle* h, const double* pos, const double* vel, const double* rho,
                  const double* drho_dt, double t, void* stream) {
  if (!h) return SPH_E_INVALID;
  Buffers& b = h->b;
  if (b.n > 0 && (!pos || !vel || !rho)) return fail(h, SPH_E_INVALID, "pos, vel and rho are required");
  if (any_foreign({pos, vel, rho, drho_dt})) return fail(h, SPH_E_INVALID, "an array lives on another device");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)b.n, d = (size_t)b.dim;
  const bool host_all = b.n >= kUploadChunkMin && !is_device_ptr(pos) && !is_device_ptr(vel) &&
                        !is_device_ptr(rho) && (!drho_dt || !is_device_ptr(drho_dt));
  if (host_all) {
    // host arrays: kUploadChunks row chunks, each imported while the next one is copied
    if (!h->up_stream) {
      CK(h, cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking));
      for (auto& e : h->up_ev) CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    double* sp = h->stage;
    double* sv = sp + n * d;
    double* sr = sv + n * d;
    double* sd = drho_dt ? sr + n : nullptr;
    CK(h, cudaEventRecord(h->up_ev[kUploadChunks], s));   // after the caller's earlier work
    CK(h, cudaStreamWaitEvent(h->up_stream, h->up_ev[kUploadChunks], 0));
    for (int c = 0; c < kUploadChunks; ++c) {
      const size_t r0 = n * c / kUploadChunks, r1 = n * (c + 1) / kUploadChunks;
      if (r1 == r0) continue;
      cudaStream_t u = h->up_stream;
      CK(h, cudaMemcpyAsync(sp + r0 * d, pos + r0 * d, sizeof(double) * (r1 - r0) * d, cudaMemcpyHostToDevice, u));
      CK(h, cudaMemcpyAsync(sv + r0 * d, vel + r0 * d, sizeof(double) * (r1 - r0) * d, cudaMemcpyHostToDevice, u));
      CK(h, cudaMemcpyAsync(sr + r0, rho + r0, sizeof(double) * (r1 - r0), cudaMemcpyHostToDevice, u));
      if (sd) CK(h, cudaMemcpyAsync(sd + r0, drho_dt + r0, sizeof(double) * (r1 - r0), cudaMemcpyHostToDevice, u));
      CK(h, cudaEventRecord(h->up_ev[c], u));
      CK(h, cudaStreamWaitEvent(s, h->up_ev[c], 0));
      sph::launch_import(b, sp, sv, sr, sd, s, (int64_t)r0, (int64_t)r1);
      ++h->launches;
    }
  } else if (b.n > 0) {
    cudaError_t e[4];
    const double* p = device_view(h, pos, n * d, 0, s, &e[0]);
    const double* v = device_view(h, vel, n * d, n * d, s, &e[1]);
    const double* r = device_view(h, rho, n, 2 * n * d, s, &e[2]);
    const double* dr = device_view(h, drho_dt, n, 2 * n * d + n, s, &e[3]);
    for (auto ee : e)
      if (ee != cudaSuccess) return cuda_fail(h, ee, "copy state");
    sph::launch_import(b, p, v, r, dr, s);
    ++h->launches;
  }
  // slot k holds caller row k until the next cell build
  sph::launch_iota(b.id, b.n, s);
  if (b.n) ++h->launches;
  sph::launch_vmax(b, s, &h->launches);
  if (t >= 0.0) {
    CK(h, cudaMemcpyAsync(&b.ctrl[0].t, &t, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  CK(h, cudaStreamSynchronize(s));          // the caller's arrays may be reused on return
  h->cells_valid = false;
  CK(h, cudaGetLastError());
  return SPH_OK;
}

int sph_build_cells(sph_handle* h, void* stream) {
  if (!h) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int r = run_build(h, s);
  if (r != SPH_OK) return r;
  h->cells_valid = true;
  return SPH_OK;
}

int sph_advection_step(sph_handle* h, double* dt_ad_out, void* stream) {
  if (!h) return SPH_E_INVALID;
  if (!h->cells_valid) return fail(h, SPH_E_INVALID, "sph_build_cells must run after a state change");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = debug_check(h, s);
  if (rc != SPH_OK) return rc;
  enqueue_advection(h, s, &h->launches);
  CK(h, cudaGetLastError());
  if (dt_ad_out) {
    CK(h, cudaMemcpyAsync(dt_ad_out, &h->b.ctrl[0].dt_ad, sizeof(double), cudaMemcpyDeviceToHost, s));
    return sync_status(h, s);
  }
  return SPH_OK;
}

int sph_acoustic_substep(sph_handle* h, int32_t* done_out, double* dt_out, void* stream) {
  if (!h) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = debug_check(h, s);
  if (rc != SPH_OK) return rc;
  enqueue_substep(h, s, false, &h->launches);
  CK(h, cudaGetLastError());
  if (done_out || dt_out || h->timing) {
    if (dt_out) CK(h, cudaMemcpyAsync(dt_out, &h->b.ctrl[0].dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    int r = sync_status(h, s);
    if (done_out) *done_out = h->hglob->active ? 0 : 1;
    if (h->timing && h->b.n > 0) {
      float a = 0.f, c = 0.f;
      cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
      cudaEventElapsedTime(&c, h->ev[1], h->ev[2]);
      h->ms[0] += a;
      h->ms[1] += c;
      h->timed[0] += 1;
      h->timed[1] += 1;
    }
    return r;
  }
  return SPH_OK;
}

int sph_step(sph_handle* h, int32_t n_advection_steps, void* stream) {
  if (!h || n_advection_steps < 0) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if ((h->flags & SPH_FLAG_PERSISTENT) && !h->timing && !debug_bounds(h) && !h->b.geo && !h->b.hrev && !h->solid) {
    // each advection step: the configuration update and the advection step's kernels, then
    // one cooperative launch for all of its substeps
    for (int k = 0; k < n_advection_steps; ++k) {
      int rb = run_build(h, s);
      if (rb != SPH_OK) return rb;
      h->cells_valid = true;
      enqueue_advection(h, s, &h->launches);
      int grid = 0;
      cudaError_t e = sph::launch_substeps_persistent(h->b, s, &grid);
      if (e != cudaSuccess) return cuda_fail(h, e, "persistent substep loop launch");
      ++h->launches;
    }
    return sync_status(h, s);
  }
  if ((h->flags & SPH_FLAG_GRAPH) && !h->timing && !debug_bounds(h)) {
    if (!h->gexec) {
      int r = build_graph(h);
      if (r != SPH_OK) return r;
    }
    CK(h, cudaMemcpyAsync(h->hglob, h->b.glob, sizeof(Global), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    long long sub0 = h->hglob->substeps;
    for (int k = 0; k < n_advection_steps; ++k) CK(h, cudaGraphLaunch(h->gexec, s));
    int r = sync_status(h, s);
    h->graph_kernels += (int64_t)n_advection_steps * h->graph_fixed +
                        (int64_t)(h->hglob->substeps - sub0) * h->graph_body;
    h->cells_valid = true;
    return r;
  }
  for (int k = 0; k < n_advection_steps; ++k) {
    int rb = run_build(h, s);
    if (rb != SPH_OK) return rb;
    h->cells_valid = true;
    enqueue_advection(h, s, &h->launches);
    for (int guard = 0;; ++guard) {
      int32_t done = 0;
      int r = sph_acoustic_substep(h, &done, nullptr, stream);
      if (r != SPH_OK) return r;
      if (done) break;
      if (guard > 1000000) return fail(h, SPH_E_UNSTABLE, "substep loop did not finish");
    }
  }
  return sync_status(h, s);
}

int sph_diagnostics(sph_handle* h, sph_diag* out, void* stream) {
  if (!h || !out) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int K = h->b.n_inst;
  sph::launch_diagnostics(h->b, h->diag_scratch, h->diag_out, s, &h->launches);
  std::vector<double> f((size_t)K * sph::kDiagFields);
  std::vector<Ctrl> c(K);
  CK(h, cudaMemcpyAsync(f.data(), h->diag_out, sizeof(double) * f.size(), cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemcpyAsync(c.data(), h->b.ctrl, sizeof(Ctrl) * K, cudaMemcpyDeviceToHost, s));
  int r = sync_status(h, s);
  for (int k = 0; k < K; ++k) {
    const double* v = &f[(size_t)k * sph::kDiagFields];
    sph_diag& d = out[k];
    std::memset(&d, 0, sizeof(d));
    d.mass = v[0];
    d.momentum[0] = v[1];
    d.momentum[1] = v[2];
    d.momentum[2] = v[3];
    d.kinetic = v[4];
    d.potential = v[5];
    d.internal = v[6];
    d.energy = v[4] + v[5] + v[6];
    d.n_fluid = (int64_t)v[10];
    d.mean_rho_dev = d.n_fluid ? v[7] / (double)d.n_fluid : 0.0;
    d.max_rho_dev = v[8];
    d.front_x = d.n_fluid ? v[9] : 0.0;
    d.t = c[k].t;
    d.dt_ad = c[k].dt_ad;
    d.advection_steps = c[k].adv_steps;
    d.substeps = c[k].substeps;
  }
  return r;
}

int sph_get_state(sph_handle* h, double* pos, double* vel, double* rho, double* drho_dt,
                  void* stream) {
  if (!h) return SPH_E_INVALID;
  Buffers& b = h->b;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)b.n, d = (size_t)b.dim;
  if (any_foreign({pos, vel, rho, drho_dt})) return fail(h, SPH_E_INVALID, "an array lives on another device");
  if (n == 0) return SPH_OK;
  double* dst[4] = {pos, vel, rho, drho_dt};
  size_t sz[4] = {n * d, n * d, n, n};
  size_t off[4] = {0, n * d, 2 * n * d, 2 * n * d + n};
  double* tgt[4];
  bool dev[4];
  for (int k = 0; k < 4; ++k) {
    dev[k] = dst[k] && is_device_ptr(dst[k]);
    tgt[k] = dst[k] ? (dev[k] ? dst[k] : h->stage + off[k]) : nullptr;
  }
  sph::launch_export(b, tgt[0], tgt[1], tgt[2], tgt[3], s);
  ++h->launches;
  for (int k = 0; k < 4; ++k)
    if (dst[k] && !dev[k])
      CK(h, cudaMemcpyAsync(dst[k], tgt[k], sizeof(double) * sz[k], cudaMemcpyDeviceToHost, s));
  return sync_status(h, s);
}

int sph_get_acceleration(sph_handle* h, double* acc, void* stream) {
  if (!h || !acc) return SPH_E_INVALID;
  if (!h->b.acc_keep) return fail(h, SPH_E_INVALID, "create the handle with SPH_FLAG_KEEP_ACC");
  if (foreign_device_ptr(acc)) return fail(h, SPH_E_INVALID, "acc lives on another device");
  cudaStream_t s = (cudaStream_t)stream;
  size_t e = (size_t)h->b.n * h->b.dim;
  bool dev = is_device_ptr(acc);
  double* tgt = dev ? acc : h->stage;
  sph::launch_export_acc(h->b, tgt, s);
  ++h->launches;
  if (!dev && e) CK(h, cudaMemcpyAsync(acc, tgt, sizeof(double) * e, cudaMemcpyDeviceToHost, s));
  return sync_status(h, s);
}

int sph_get_permutation(sph_handle* h, int32_t* ids, void* stream) {
  if (!h || !ids) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->b.n) CK(h, cudaMemcpyAsync(ids, h->b.id, sizeof(int) * h->b.n, cudaMemcpyDefault, s));
  return sync_status(h, s);
}

int sph_get_neighbours(sph_handle* h, int32_t* fluid_count, int32_t* wall_count, int32_t* fluid_ids,
                       int32_t* wall_ids, int32_t stride, void* stream) {
  if (!h || !fluid_count || !wall_count || !fluid_ids || !wall_ids) return SPH_E_INVALID;
  if (stride < h->b.cap) return fail(h, SPH_E_INVALID, "stride must be >= capacity");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = debug_check(h, s);
  if (rc != SPH_OK) return rc;
  const size_t n = (size_t)h->b.n;
  if (n == 0) return SPH_OK;
  int32_t *fc, *wc, *fi, *wi;
  CK(h, cudaMalloc(&fc, sizeof(int32_t) * n));
  CK(h, cudaMalloc(&wc, sizeof(int32_t) * n));
  CK(h, cudaMalloc(&fi, sizeof(int32_t) * n * stride));
  CK(h, cudaMalloc(&wi, sizeof(int32_t) * n * stride));
  sph::launch_export_neighbours(h->b, fc, wc, fi, wi, stride, s);
  ++h->launches;
  cudaMemcpyAsync(fluid_count, fc, sizeof(int32_t) * n, cudaMemcpyDefault, s);
  cudaMemcpyAsync(wall_count, wc, sizeof(int32_t) * n, cudaMemcpyDefault, s);
  cudaMemcpyAsync(fluid_ids, fi, sizeof(int32_t) * n * stride, cudaMemcpyDefault, s);
  cudaMemcpyAsync(wall_ids, wi, sizeof(int32_t) * n * stride, cudaMemcpyDefault, s);
  int r = sync_status(h, s);
  cudaFree(fc);
  cudaFree(wc);
  cudaFree(fi);
  cudaFree(wi);
  return r;
}

int sph_pair_count(sph_handle* h, int64_t* fluid_pairs, int64_t* wall_pairs, void* stream) {
  if (!h || !fluid_pairs || !wall_pairs) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = debug_check(h, s);
  if (rc != SPH_OK) return rc;
  unsigned long long* d = reinterpret_cast<unsigned long long*>(h->diag_out);
  unsigned long long hv[2] = {0, 0};
  sph::launch_pair_count(h->b, d, s);
  ++h->launches;
  CK(h, cudaMemcpyAsync(hv, d, sizeof(hv), cudaMemcpyDeviceToHost, s));
  int r = sync_status(h, s);
  *fluid_pairs = (int64_t)hv[0];
  *wall_pairs = (int64_t)hv[1];
  return r;
}

int sph_get_launch_config(const sph_handle* h, int32_t* cfg) {
  if (!h || !cfg) return SPH_E_INVALID;
  cfg[0] = h->b.cfg.pr_tpp;
  cfg[1] = h->b.cfg.pr_block;
  cfg[2] = h->b.cfg.dr_tpp;
  cfg[3] = h->b.cfg.dr_block;
  return SPH_OK;
}

int sph_set_gravity(sph_handle* h, int32_t instance, const double* g, void* stream) {
  if (!h) return SPH_E_INVALID;
  if (!g) return fail(h, SPH_E_INVALID, "g is required");
  const int n_inst = h->b.n_inst, d = h->b.dim;
  if (instance >= n_inst) return fail(h, SPH_E_INVALID, "no such tank");
  for (int a = 0; a < d; ++a)
    if (!std::isfinite(g[a])) return fail(h, SPH_E_INVALID, "gravity must be finite");
  cudaStream_t s = (cudaStream_t)stream;
  const int k0 = instance < 0 ? 0 : instance, k1 = instance < 0 ? n_inst : instance + 1;
  for (int k = k0; k < k1; ++k) {
    for (int a = 0; a < 3; ++a) {
      h->params[k].gravity[a] = a < d ? g[a] : 0.0;
      h->hinst[k].g[a] = a < d ? (float)g[a] : 0.0f;
    }
    // the device copy, in stream order with the work already queued
    CK(h, cudaMemcpyAsync(h->b.inst + k, &h->hinst[k], sizeof(Inst), cudaMemcpyHostToDevice, s));
  }
  h->b.inst0 = h->hinst[0];
  if (k0 == 0) sph_fsi_set_gravity(h, h->params[0].gravity);   // a solid lives in tank 0
  drop_graph(h);
  CK(h, cudaStreamSynchronize(s));                 // the host copies above are read now
  return SPH_OK;
}

int sph_set_launch_config(sph_handle* h, const int32_t* cfg) {
  if (!h || !cfg) return SPH_E_INVALID;
  std::ostringstream o;
  o << cfg[0] << "," << cfg[1] << "," << cfg[2] << "," << cfg[3];
  sph::LaunchCfg c;
  if (!parse_cfg(o.str(), &c, h->b.n_inst == 1))
    return fail(h, SPH_E_INVALID, "threads per particle must be 1, 2 or 4 and blocks 128, 256 or 512, or 1 and 896 "
                                  "(row tasks, one tank)");
  h->b.cfg = c;
  drop_graph(h);
  return SPH_OK;
}

int sph_autotune(sph_handle* h, int32_t* cfg_out, double* ms_out, void* stream) {
  if (!h) return SPH_E_INVALID;
  if (h->b.hrev) return fail(h, SPH_E_INVALID, "the half-pair evaluation has no launch variants to tune");
  cudaStream_t s = (cudaStream_t)stream;
  int rb = run_build(h, s);
  if (rb != SPH_OK) return rb;
  h->cells_valid = true;
  enqueue_advection(h, s, &h->launches);
  sph::launch_dt_acoustic(h->b, s, h->cond, false, &h->launches);
  cudaEvent_t e0 = h->ev[0], e1 = h->ev[1];
  const int reps = 3;
  // the row-task form is a tenth variant of each kernel on handles of one tank
  const bool rows = h->b.row_task && !h->b.geo;
  if (rows && !h->rows_valid) {
    sph::launch_row_tasks(h->b, s, &h->launches);
    h->rows_valid = true;
  }
  // repeated launches of either kernel are idempotent: same inputs, same outputs
  for (int kernel = 0; kernel < 2; ++kernel) {
    float best = 1e30f;
    sph::LaunchCfg best_cfg = h->b.cfg;
    for (int v = 0; v < kAutotuneVariants; ++v) {
      const int t = v < 9 ? kTppChoices[v / 3] : 1, blk = v < 9 ? kBlockChoices[v % 3] : sph::kRowBlock;
      if (v == 9 && !rows) {
        if (ms_out) ms_out[kernel * kAutotuneVariants + v] = -1.0;   // not available
        continue;
      }
      sph::LaunchCfg c = h->b.cfg;
      if (kernel == 0) { c.pr_tpp = t; c.pr_block = blk; } else { c.dr_tpp = t; c.dr_block = blk; }
      sph::Buffers bb = h->b;
      bb.cfg = c;
      CK(h, cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r) {
        if (kernel == 0) sph::launch_pressure_relaxation(bb, s, &h->launches);
        else sph::launch_density_relaxation(bb, s, &h->launches);
      }
      CK(h, cudaEventRecord(e1, s));
      CK(h, cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(h, cudaEventElapsedTime(&ms, e0, e1));
      ms /= reps;
      if (ms_out) ms_out[kernel * kAutotuneVariants + v] = ms;
      if (ms < best) {
        best = ms;
        best_cfg = c;
      }
    }
    h->b.cfg = best_cfg;
    // the stored result comes from the chosen variant
    if (kernel == 0) sph::launch_pressure_relaxation(h->b, s, &h->launches);
    else sph::launch_density_relaxation(h->b, s, &h->launches);
  }
  drop_graph(h);
  int r = sync_status(h, s);
  if (r != SPH_OK) return r;
  // finish the advection step with the chosen configuration
  for (int guard = 0; h->hglob->active; ++guard) {
    int32_t done = 0;
    r = sph_acoustic_substep(h, &done, nullptr, stream);
    if (r != SPH_OK) return r;
    if (done) break;
    if (guard > 1000000) return fail(h, SPH_E_UNSTABLE, "substep loop did not finish");
  }
  auto cache = read_autotune_cache();
  cache[autotune_key(h)] = format_cfg(h->b.cfg);
  write_autotune_cache(cache);
  if (cfg_out) sph_get_launch_config(h, cfg_out);
  return SPH_OK;
}

int sph_gather_ceiling(sph_handle* h, int32_t reps, double* ms_out, void* stream) {
  if (!h || !ms_out || reps < 1) return SPH_E_INVALID;
  if (!h->cells_valid) return fail(h, SPH_E_INVALID, "sph_build_cells must run first");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = debug_check(h, s);
  if (rc != SPH_OK) return rc;
  unsigned* sink = reinterpret_cast<unsigned*>(h->diag_out);
  sph::launch_gather_ceiling(h->b, sink, s, &h->launches);        // warm-up
  CK(h, cudaEventRecord(h->ev[0], s));
  for (int r = 0; r < reps; ++r) sph::launch_gather_ceiling(h->b, sink, s, &h->launches);
  CK(h, cudaEventRecord(h->ev[1], s));
  CK(h, cudaEventSynchronize(h->ev[1]));
  float ms = 0.f;
  CK(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
  *ms_out = (double)ms / reps;
  return sync_status(h, s);
}

int sph_clear_error(sph_handle* h, void* stream) {
  if (!h) return SPH_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  CK(h, cudaMemsetAsync(&h->b.glob->err, 0, sizeof(int), s));
  CK(h, cudaMemsetAsync(&h->b.glob->bad_index, 0, sizeof(long long), s));
  CK(h, cudaStreamSynchronize(s));
  h->err.clear();
  return SPH_OK;
}

int sph_debug_write(sph_handle* h, int32_t what, int64_t index, int32_t slot, int64_t value, void* stream) {
  if (!h) return SPH_E_INVALID;
  if (!debug_bounds(h)) return fail(h, SPH_E_INVALID, "sph_debug_write needs a handle created with SPH_FLAG_DEBUG_BOUNDS");
  cudaStream_t s = (cudaStream_t)stream;
  const Buffers& b = h->b;
  if (what == SPH_DEBUG_NEIGHBOUR) {
    if (index < 0 || index >= b.n || slot < 0 || slot >= b.cap)
      return fail(h, SPH_E_INVALID, "sph_debug_write: row or slot out of range");
    const int v = (int)value;
    const int64_t at = ((int64_t)(slot >> 2) * b.n + index) * 4 + (slot & 3);
    CK(h, cudaMemcpyAsync(b.nbr + at, &v, sizeof(int), cudaMemcpyHostToDevice, s));
  } else if (what == SPH_DEBUG_WALL_OFFSET) {
    if (index < 0 || index > b.n_cells) return fail(h, SPH_E_INVALID, "sph_debug_write: cell out of range");
    const uint32_t v = (uint32_t)value;
    CK(h, cudaMemcpyAsync(b.wstart + index, &v, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  } else {
    return fail(h, SPH_E_INVALID, "sph_debug_write: unknown table");
  }
  CK(h, cudaStreamSynchronize(s));
  return SPH_OK;
}

int sph_kernel_launches(sph_handle* h, int64_t* out) {
  if (!h || !out) return SPH_E_INVALID;
  *out = h->launches + h->graph_kernels;
  return SPH_OK;
}

int sph_set_kernel_timing(sph_handle* h, int32_t enable) {
  if (!h) return SPH_E_INVALID;
  h->timing = enable != 0;
  h->ms[0] = h->ms[1] = 0.0;
  h->timed[0] = h->timed[1] = 0;
  return SPH_OK;
}

int sph_kernel_times(sph_handle* h, double* ms, int64_t* launches) {
  if (!h) return SPH_E_INVALID;
  if (ms) {
    ms[0] = h->ms[0];
    ms[1] = h->ms[1];
  }
  if (launches) {
    launches[0] = h->timed[0];
    launches[1] = h->timed[1];
  }
  return SPH_OK;
}

}  // extern "C"

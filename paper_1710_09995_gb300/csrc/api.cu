// api.cu -- the C ABI declared in include/gbcfd.h.
//
// A block is a host descriptor plus arrays carved from caller device memory.  Every call is
// enqueued on the caller's stream; only residual_norm / get_dt / get_state-to-host wait.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gbcfd.h"
#include "launch.h"
#include "learn.cuh"

using namespace gbcfd;

// ---- error state ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
static int cuda_fail(cudaError_t e, const char* what) {
  return fail(GBCFD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

extern "C" const char* gbcfd_last_error(void) { return g_err.c_str(); }

int gbcfd::set_error(int code, const std::string& msg) { return fail(code, msg); }

// ---- block descriptor ----------------------------------------------------------------------
struct gbcfd_block_s {
  int nx, ny, nz;
  gbcfd_params p;
  Geometry g;
  int device, nsm, grid;
  size_t bytes;
  double* q[3];      // FP64: Qn, Q1, Q2.  mixed: QA, QB (ping-pong Q^n)
  float* sh[2];      // mixed: SA, SB, the f32 shadows of QA, QB
  float* d[2];       // mixed: D1, D2
  void* metrics;     // 10 fields (f64, or f32 on the mixed path)
  DevCtrl* ctrl;
  double* partial;
  char* staging;     // host-transfer staging (aliases the stage buffers)
  size_t staging_bytes;
  int cur;           // mixed: index of Q^n in q[]
  int has_state;
  int next_stage;    // 1, 2 or 3: the Runge-Kutta stage the block expects next
  double spacing[3];
  gbcfd_block nbr[6];
  CUtensorMap tm_q[3];  // FP64: maps of Qn, Q1, Q2.  mixed: maps of the shadows SA, SB
  CUtensorMap tm_d[2];
  CUtensorMap tm_m;     // metric planes (10 fields)
  BlockDesc* desc;      // the block's descriptor in device memory (a group of one)
  BlockDesc desc_host;  // host copy
  int curvi;            // metrics from nodes (curvilinear) rather than a uniform spacing
  int metrics_dirty;    // metric halos not exchanged since the metrics were set
  void* dtl;            // local time steps (local_dt), one padded field of the path's flux type
  unsigned desc_version;  // bumped whenever the device descriptor changes
  int bc_kind[6];       // GBCFD_BC_* per face (faces without a neighbour)
  double bc_inf[5];     // free stream of GBCFD_BC_FARFIELD faces
};

static int prepare_metrics(const gbcfd_block* blocks, int n, cudaStream_t s);
static int init_rate(gbcfd_block b, cudaStream_t s);

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int pitch_for(int nx, int elem) {
  const int per = 128 / elem;  // 128-byte rows
  return (nx + 2 * HALO + per - 1) / per * per;
}

static Geometry make_geometry(int nx, int ny, int nz) {
  Geometry g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.px = pitch_for(nx, 8);
  g.pxf = pitch_for(nx, 4);
  g.plane = (long long)(ny + 2 * HALO) * g.px;
  g.planef = (long long)(ny + 2 * HALO) * g.pxf;
  g.field = g.plane * (nz + 2 * HALO);
  g.fieldf = g.planef * (nz + 2 * HALO);
  return g;
}

static bool valid_params(const gbcfd_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (!(p->gamma > 1.0)) { why = "gamma must be > 1"; return false; }
  if (!(p->cfl > 0.0)) { why = "cfl must be > 0"; return false; }
  if (!(p->entropy_eps >= 0.0)) { why = "entropy_eps must be >= 0"; return false; }
  if (p->viscous && !(p->mu >= 0.0 && p->Pr > 0.0)) { why = "viscous needs mu >= 0 and Pr > 0"; return false; }
  if (p->limiter != 0 && p->limiter != 1) { why = "limiter must be 0 or 1"; return false; }
  if (p->precision != GBCFD_FP64 && p->precision != GBCFD_MIXED) { why = "bad precision"; return false; }
  if (p->local_dt != 0 && p->local_dt != 1) { why = "local_dt must be 0 or 1"; return false; }
  if (p->local_dt && p->viscous) { why = "local time steps are for inviscid blocks (viscous = 0)"; return false; }
  return true;
}

// stage grid: resident CTAs on every SM, capped by the number of tile-planes
static int stage_grid(const Geometry& g, int precision, int viscous, int curvi, int nsm) {
  const int occ = precision == GBCFD_MIXED ? (curvi ? stage_occupancy_f32c(viscous) : stage_occupancy_f32(viscous))
                                           : (curvi ? stage_occupancy_f64c(viscous) : stage_occupancy_f64(viscous));
  const long long units = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY_DEFAULT - 1) / TY_DEFAULT) * g.nz;
  long long grid = (long long)nsm * occ;
  if (grid > units) grid = units;
  return (int)std::max(1LL, grid);
}

struct Carve {
  size_t off[12];
  size_t total;
  size_t partial_n;
};

static Carve carve(const Geometry& g, int precision, int local_dt, int nsm) {
  Carve c;
  size_t o = 0;
  const size_t f64 = align256(sizeof(double) * 5 * g.field);
  const size_t f32 = align256(sizeof(float) * 5 * g.fieldf);
  c.off[0] = o; o += f64;                   // q0
  c.off[1] = o; o += f64;                   // q1
  if (precision == GBCFD_FP64) {
    c.off[2] = o; o += f64;                 // q2
    c.off[3] = c.off[4] = 0;
    c.off[5] = o; o += align256(sizeof(double) * 10 * g.field);  // metrics f64
  } else {
    c.off[2] = 0;
    c.off[3] = o; o += f32;                 // d0
    c.off[4] = o; o += f32;                 // d1
    c.off[5] = o; o += align256(sizeof(float) * 10 * g.fieldf);  // metrics f32
    c.off[8] = o; o += f32;                 // shadow A
    c.off[9] = o; o += f32;                 // shadow B
  }
  c.off[6] = o; o += align256(sizeof(DevCtrl));
  c.off[10] = o; o += align256(sizeof(BlockDesc));
  c.partial_n = (size_t)std::max(4 * nsm, 4 * 152);
  c.off[7] = o; o += align256(sizeof(double) * NPART * c.partial_n);
  c.off[11] = 0;
  if (local_dt) {  // one padded field of local time steps
    c.off[11] = o;
    o += precision == GBCFD_FP64 ? align256(sizeof(double) * g.field) : align256(sizeof(float) * g.fieldf);
  }
  c.total = o;
  return c;
}

static int device_sms(int* dev, int* nsm) {
  CK(cudaGetDevice(dev));
  CK(cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, *dev));
  return GBCFD_OK;
}

// ---- TMA descriptors -------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 4D map (x, y, z, variable) over a padded field; box = one tile plane with its halo (rows: the
// tile height + 4), all nvar variables.  x extent is the padded width nx + 4, so a box past it is
// zero-filled.  No L2 promotion: a box row is 36 values from a 128-byte boundary, and 256-byte
// promotion fetched up to 512 bytes of DRAM for it (measured at 256^3: 15-20% more DRAM reads per
// launch for the same time).
static int make_map(CUtensorMap* m, void* base, const Geometry& g, int elem, int nvar = 5,
                    int rows = box_rows(TY_DEFAULT)) {
  auto enc = get_encode();
  if (!enc) return fail(GBCFD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const int pitch = elem == 8 ? g.px : g.pxf;
  cuuint64_t dims[4] = {(cuuint64_t)(g.nx + 2 * HALO), (cuuint64_t)(g.ny + 2 * HALO),
                        (cuuint64_t)(g.nz + 2 * HALO), (cuuint64_t)nvar};
  cuuint64_t strides[3] = {(cuuint64_t)pitch * elem, (cuuint64_t)pitch * elem * (g.ny + 2 * HALO),
                           (cuuint64_t)pitch * elem * (g.ny + 2 * HALO) * (g.nz + 2 * HALO)};
  cuuint32_t box[4] = {(cuuint32_t)BX, (cuuint32_t)rows, 1, (cuuint32_t)nvar};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base,
                   dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GBCFD_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return GBCFD_OK;
}

// ---- creation --------------------------------------------------------------------------------
extern "C" int gbcfd_required_bytes(int nx, int ny, int nz, const gbcfd_params* params, size_t* bytes) {
  std::string why;
  if (nx < 1 || ny < 1 || nz < 1) return fail(GBCFD_ERR_ARG, "block sizes must be >= 1");
  if (!bytes) return fail(GBCFD_ERR_ARG, "bytes is NULL");
  if (!valid_params(params, why)) return fail(GBCFD_ERR_ARG, why);
  int dev = 0, nsm = 152;
  int rc = device_sms(&dev, &nsm);
  if (rc) return rc;
  *bytes = carve(make_geometry(nx, ny, nz), params->precision, params->local_dt, nsm).total;
  return GBCFD_OK;
}

static Physics physics_of(const gbcfd_block_s* b) {
  Physics ph;
  ph.gamma = b->p.gamma;
  ph.mu = b->p.mu;
  ph.Pr = b->p.Pr;
  ph.cfl = b->p.cfl;
  ph.eps = b->p.entropy_eps;
  ph.ihx = 1.0 / b->spacing[0];
  ph.ihy = 1.0 / b->spacing[1];
  ph.ihz = 1.0 / b->spacing[2];
  ph.viscous = b->p.viscous;
  ph.limiter = b->p.limiter;
  ph.local_dt = b->p.local_dt;
  return ph;
}

// the stage kernel's constants in both precisions (formed here, once)
template <typename T>
static PathK<T> path_k_of(const Physics& ph) {
  PathK<T> k;
  const double kappa = ph.Pr > 0.0 ? ph.mu * ph.gamma / ((ph.gamma - 1.0) * ph.Pr) : 0.0;
  k.gm1 = T(ph.gamma - 1.0);
  k.ggm1 = T(ph.gamma / (ph.gamma - 1.0));
  k.eps = T(ph.eps);
  k.mu = T(ph.mu);
  k.kappa = T(kappa);
  k.gam = T(ph.gamma);
  k.vf = T(4.0 * std::max(4.0 / 3.0, ph.gamma / ph.Pr) * ph.mu);
  k.cfl = T(ph.cfl);
  return k;
}
static PathConsts path_consts(const Physics& ph) {
  PathConsts c;
  c.f = path_k_of<float>(ph);
  c.d = path_k_of<double>(ph);
  return c;
}

// the block as the stage kernel sees it
static void fill_desc(gbcfd_block_s* b) {
  BlockDesc& D = b->desc_host;
  memset(&D, 0, sizeof(D));
  for (int i = 0; i < 3; ++i) D.tq[i] = b->tm_q[i];
  for (int i = 0; i < 2; ++i) D.td[i] = b->tm_d[i];
  D.tm = b->tm_m;
  D.g = b->g;
  D.ihx = 1.0 / b->spacing[0];
  D.ihy = 1.0 / b->spacing[1];
  D.ihz = 1.0 / b->spacing[2];
  D.ihxf = (float)D.ihx;
  D.ihyf = (float)D.ihy;
  D.ihzf = (float)D.ihz;
  for (int i = 0; i < 3; ++i) D.q[i] = b->q[i];
  for (int i = 0; i < 2; ++i) { D.sh[i] = b->sh[i]; D.d[i] = b->d[i]; }
  D.ctrl = b->ctrl;
  D.dtl = b->dtl;
  b->desc_version++;
  D.ntx = (b->nx + TX - 1) / TX;
  D.nty = (b->ny + TY_DEFAULT - 1) / TY_DEFAULT;
  D.units = (long long)D.ntx * D.nty * b->nz;
  D.cta0 = 0;
  D.ctas = b->grid;
}

// the block's descriptor for a stage kernel compiled with tile height ty: the default one, or a
// copy whose tensor maps move (ty + 4)-row boxes and whose tile counts use ty
static int write_desc(const gbcfd_block_s* b, int ty, BlockDesc* D) {
  *D = b->desc_host;
  if (ty == TY_DEFAULT) return GBCFD_OK;
  const int rows = box_rows(ty);
  int r = GBCFD_OK;
  if (b->p.precision == GBCFD_FP64) {
    for (int i = 0; i < 3 && !r; ++i) r = make_map(&D->tq[i], b->q[i], b->g, 8, 5, rows);
    if (!r) D->td[0] = D->td[1] = D->tq[0];
  } else {
    for (int i = 0; i < 2 && !r; ++i) r = make_map(&D->tq[i], b->sh[i], b->g, 4, 5, rows);
    for (int i = 0; i < 2 && !r; ++i) r = make_map(&D->td[i], b->d[i], b->g, 4, 5, rows);
    if (!r) D->tq[2] = D->tq[0];
  }
  if (!r && b->curvi) r = make_map(&D->tm, b->metrics, b->g, b->p.precision == GBCFD_MIXED ? 4 : 8, 10, rows);
  if (r) return r;
  D->nty = (b->ny + ty - 1) / ty;
  D->units = (long long)D->ntx * D->nty * b->nz;
  return GBCFD_OK;
}

extern "C" int gbcfd_create_block(int nx, int ny, int nz, const gbcfd_params* params, void* dev_mem,
                                  size_t bytes, gbcfd_block* out) {
  std::string why;
  if (!out) return fail(GBCFD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(GBCFD_ERR_ARG, "block sizes must be >= 1");
  if (!valid_params(params, why)) return fail(GBCFD_ERR_ARG, why);
  if (!dev_mem) return fail(GBCFD_ERR_ARG, "dev_mem is NULL");
  if (((uintptr_t)dev_mem & 255u) != 0) return fail(GBCFD_ERR_MEMORY, "dev_mem must be 256-byte aligned");
  cudaPointerAttributes attr;
  CK(cudaPointerGetAttributes(&attr, dev_mem));
  if (attr.type != cudaMemoryTypeDevice) return fail(GBCFD_ERR_MEMORY, "dev_mem is not device memory");
  int dev = 0, nsm = 0;
  int rc = device_sms(&dev, &nsm);
  if (rc) return rc;
  Geometry g = make_geometry(nx, ny, nz);
  Carve c = carve(g, params->precision, params->local_dt, nsm);
  if (bytes < c.total) return fail(GBCFD_ERR_MEMORY, "dev_mem smaller than gbcfd_required_bytes");

  gbcfd_block_s* b = new gbcfd_block_s();
  b->nx = nx; b->ny = ny; b->nz = nz;
  b->p = *params;
  b->g = g;
  b->device = dev;
  b->nsm = nsm;
  b->bytes = bytes;
  char* base = static_cast<char*>(dev_mem);
  b->q[0] = reinterpret_cast<double*>(base + c.off[0]);
  b->q[1] = reinterpret_cast<double*>(base + c.off[1]);
  b->q[2] = params->precision == GBCFD_FP64 ? reinterpret_cast<double*>(base + c.off[2]) : nullptr;
  b->d[0] = params->precision == GBCFD_MIXED ? reinterpret_cast<float*>(base + c.off[3]) : nullptr;
  b->d[1] = params->precision == GBCFD_MIXED ? reinterpret_cast<float*>(base + c.off[4]) : nullptr;
  b->sh[0] = params->precision == GBCFD_MIXED ? reinterpret_cast<float*>(base + c.off[8]) : nullptr;
  b->sh[1] = params->precision == GBCFD_MIXED ? reinterpret_cast<float*>(base + c.off[9]) : nullptr;
  b->metrics = base + c.off[5];
  b->ctrl = reinterpret_cast<DevCtrl*>(base + c.off[6]);
  b->partial = reinterpret_cast<double*>(base + c.off[7]);
  b->dtl = params->local_dt ? static_cast<void*>(base + c.off[11]) : nullptr;
  b->desc_version = 0;
  for (int f = 0; f < 6; ++f) b->bc_kind[f] = GBCFD_BC_NONE;
  for (int v = 0; v < 5; ++v) b->bc_inf[v] = 0.0;
  if (params->precision == GBCFD_FP64) {
    b->staging = reinterpret_cast<char*>(b->q[1]);
    b->staging_bytes = c.off[2] - c.off[1];
  } else {
    b->staging = reinterpret_cast<char*>(b->d[0]);
    b->staging_bytes = c.off[5] - c.off[3];
  }
  b->cur = 0;
  b->has_state = 0;
  b->next_stage = 1;
  b->spacing[0] = b->spacing[1] = b->spacing[2] = 1.0;
  for (int f = 0; f < 6; ++f) b->nbr[f] = nullptr;
  b->curvi = 0;
  b->metrics_dirty = 0;
  b->grid = stage_grid(g, params->precision, params->viscous, 0, nsm);
  if ((size_t)b->grid > c.partial_n) b->grid = (int)c.partial_n;

  int r = GBCFD_OK;
  if (params->precision == GBCFD_FP64) {
    for (int i = 0; i < 3 && !r; ++i) r = make_map(&b->tm_q[i], b->q[i], g, 8);
    if (!r) b->tm_d[0] = b->tm_d[1] = b->tm_q[0];
  } else {
    for (int i = 0; i < 2 && !r; ++i) r = make_map(&b->tm_q[i], b->sh[i], g, 4);
    for (int i = 0; i < 2 && !r; ++i) r = make_map(&b->tm_d[i], b->d[i], g, 4);
    if (!r) b->tm_q[2] = b->tm_q[0];
  }
  if (!r) r = make_map(&b->tm_m, b->metrics, g, params->precision == GBCFD_MIXED ? 4 : 8, 10);
  if (r) { delete b; return r; }
  b->desc = reinterpret_cast<BlockDesc*>(base + c.off[10]);
  fill_desc(b);
  cudaError_t e = cudaMemset(b->ctrl, 0, sizeof(DevCtrl));
  if (e == cudaSuccess) e = cudaMemcpy(b->desc, &b->desc_host, sizeof(BlockDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "initialising the block"); }
  *out = b;
  return GBCFD_OK;
}

extern "C" int gbcfd_destroy_block(gbcfd_block b) {
  if (!b) return fail(GBCFD_ERR_ARG, "block is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  delete b;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  return GBCFD_OK;
}

extern "C" int gbcfd_connect(gbcfd_block b, int face, gbcfd_block nbr) {
  if (!b || !nbr) return fail(GBCFD_ERR_ARG, "block is NULL");
  if (face < 0 || face > 5) return fail(GBCFD_ERR_ARG, "face must be 0..5");
  const int d = face / 2;
  const int na[3] = {b->nx, b->ny, b->nz}, nb[3] = {nbr->nx, nbr->ny, nbr->nz};
  for (int a = 0; a < 3; ++a)
    if (a != d && na[a] != nb[a]) return fail(GBCFD_ERR_ARG, "connected faces must have equal cell counts");
  if (b->p.precision != nbr->p.precision) return fail(GBCFD_ERR_ARG, "connected blocks must share a precision");
  if (b->bc_kind[face] != GBCFD_BC_NONE || nbr->bc_kind[face ^ 1] != GBCFD_BC_NONE)
    return fail(GBCFD_ERR_ARG, "a face with a boundary condition cannot be connected");
  b->nbr[face] = nbr;
  nbr->nbr[face ^ 1] = b;
  return GBCFD_OK;
}

extern "C" int gbcfd_set_boundary(gbcfd_block b, int face, int kind, const double inf[5]) {
  if (!b) return fail(GBCFD_ERR_ARG, "block is NULL");
  if (face < 0 || face > 5) return fail(GBCFD_ERR_ARG, "face must be 0..5");
  if (kind != GBCFD_BC_NONE && kind != GBCFD_BC_SLIP_WALL && kind != GBCFD_BC_FARFIELD)
    return fail(GBCFD_ERR_ARG, "unknown boundary kind");
  if (kind != GBCFD_BC_NONE) {
    if (b->nbr[face]) return fail(GBCFD_ERR_ARG, "the face is connected to a neighbour");
    if (b->p.viscous) return fail(GBCFD_ERR_ARG, "boundary conditions are inviscid: the block must have viscous = 0");
    const int n[3] = {b->nx, b->ny, b->nz};
    if (n[face / 2] < 2) return fail(GBCFD_ERR_ARG, "a boundary face needs at least 2 cells across the block");
  }
  if (kind == GBCFD_BC_FARFIELD) {
    if (!inf) return fail(GBCFD_ERR_ARG, "a far-field face needs the free stream");
    if (!(inf[0] > 0.0 && inf[4] > 0.0) || !std::isfinite(inf[1]) || !std::isfinite(inf[2]) || !std::isfinite(inf[3]))
      return fail(GBCFD_ERR_ARG, "the free stream needs rho > 0, p > 0 and a finite velocity");
    for (int v = 0; v < 5; ++v) b->bc_inf[v] = inf[v];
  }
  b->bc_kind[face] = kind;
  return GBCFD_OK;
}

extern "C" int gbcfd_set_metrics(gbcfd_block b, const double* nodes, const double spacing[3], void* stream) {
  if (!b) return fail(GBCFD_ERR_ARG, "block is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!nodes) {
    if (!spacing || !(spacing[0] > 0 && spacing[1] > 0 && spacing[2] > 0))
      return fail(GBCFD_ERR_ARG, "spacing must be three positive cell sizes");
    for (int a = 0; a < 3; ++a) b->spacing[a] = spacing[a];
    if (b->curvi) {
      b->curvi = 0;
      b->metrics_dirty = 0;
      b->grid = stage_grid(b->g, b->p.precision, b->p.viscous, 0, b->nsm);
    }
    fill_desc(b);
    CK(cudaMemcpy(b->desc, &b->desc_host, sizeof(BlockDesc), cudaMemcpyHostToDevice));
    return GBCFD_OK;
  }
  cudaPointerAttributes attr;
  CK(cudaPointerGetAttributes(&attr, nodes));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(GBCFD_ERR_ARG, "nodes must be device memory");
  CK(launch_metrics(b->g, nodes, b->metrics, b->p.precision == GBCFD_MIXED ? 4 : 8, s));
  b->curvi = 1;
  b->metrics_dirty = 1;
  b->grid = stage_grid(b->g, b->p.precision, b->p.viscous, 1, b->nsm);
  fill_desc(b);
  CK(cudaMemcpy(b->desc, &b->desc_host, sizeof(BlockDesc), cudaMemcpyHostToDevice));
  return GBCFD_OK;
}

// ---- state in / out ------------------------------------------------------------------------
// where a caller's array lives: *dev for device (or managed) memory; otherwise *mapped is the
// device address of pinned host memory (the GPU reads and writes it over the host link with the
// same pointer under unified addressing), or NULL for pageable memory (copied through staging)
static int locate_ptr(const void* p, bool* dev, void** mapped) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
  *dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  *mapped = (!*dev && a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
  return GBCFD_OK;
}
static int is_device_ptr(const void* p, bool* dev) {
  void* mapped = nullptr;
  return locate_ptr(p, dev, &mapped);
}

static double* state_ptr(gbcfd_block b) {
  return b->p.precision == GBCFD_FP64 ? b->q[0] : b->q[b->cur];
}

extern "C" int gbcfd_set_state(gbcfd_block b, const double* q, void* stream) {
  if (!b || !q) return fail(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)b->nx * b->ny * b->nz;
  bool dev = false;
  void* mapped = nullptr;
  int rc = locate_ptr(q, &dev, &mapped);
  if (rc) return rc;
  const double* src = q;
  if (!dev && mapped) {
    src = static_cast<const double*>(mapped);  // pinned host memory: the scatter reads it directly
  } else if (!dev) {
    if (b->staging_bytes < 5 * n * sizeof(double)) return fail(GBCFD_ERR_MEMORY, "staging too small");
    CK(cudaMemcpyAsync(b->staging, q, 5 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    src = reinterpret_cast<const double*>(b->staging);
  }
  CK(launch_scatter(b->g, src, state_ptr(b), b->p.precision == GBCFD_MIXED ? b->sh[b->cur] : nullptr, s));
  b->has_state = 1;
  b->next_stage = 1;
  if (b->metrics_dirty) return prepare_metrics(&b, 1, s);  // also evaluates the time step
  return init_rate(b, s);
}

extern "C" int gbcfd_get_state(gbcfd_block b, double* q, void* stream) {
  if (!b || !q) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (!b->has_state) return fail(GBCFD_ERR_STATE, "no state set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)b->nx * b->ny * b->nz;
  bool dev = false;
  void* mapped = nullptr;
  int rc = locate_ptr(q, &dev, &mapped);
  if (rc) return rc;
  if (dev) {
    CK(launch_gather(b->g, state_ptr(b), q, s));
    return GBCFD_OK;
  }
  if (mapped) {  // pinned host memory: the gather writes it directly
    CK(launch_gather(b->g, state_ptr(b), static_cast<double*>(mapped), s));
    CK(cudaStreamSynchronize(s));
    return GBCFD_OK;
  }
  double* tmp = reinterpret_cast<double*>(b->staging);
  CK(launch_gather(b->g, state_ptr(b), tmp, s));
  CK(cudaMemcpyAsync(q, tmp, 5 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GBCFD_OK;
}

// ---- halo exchange over a group -----------------------------------------------------------
enum Field { F_STATE = 0, F_STAGE1 = 1, F_STAGE2 = 2, F_METRICS = 3 };

static void field_of(gbcfd_block b, int f, char** base, int* elem, int* nvar) {
  const bool mixed = b->p.precision == GBCFD_MIXED;
  *nvar = 5;
  switch (f) {
    case F_STATE:  // the mixed path's stencils read the f32 shadow of Q^n
      *base = mixed ? reinterpret_cast<char*>(b->sh[b->cur]) : reinterpret_cast<char*>(state_ptr(b));
      *elem = mixed ? 4 : 8;
      break;
    case F_STAGE1: *base = mixed ? reinterpret_cast<char*>(b->d[0]) : reinterpret_cast<char*>(b->q[1]); *elem = mixed ? 4 : 8; break;
    case F_STAGE2: *base = mixed ? reinterpret_cast<char*>(b->d[1]) : reinterpret_cast<char*>(b->q[2]); *elem = mixed ? 4 : 8; break;
    default: *base = reinterpret_cast<char*>(b->metrics); *elem = mixed ? 4 : 8; *nvar = 10; break;
  }
}

// fills halos of blocks[0..n); neighbours outside the list are read as sources when
// allow_external, else the call fails
static int build_group(const gbcfd_block* blocks, int n, int field, bool allow_external, HaloGroup* G) {
  std::vector<gbcfd_block> list(blocks, blocks + n);
  for (size_t i = 0; i < list.size(); ++i) {
    for (int f = 0; f < 6; ++f) {
      gbcfd_block nb = list[i]->nbr[f];
      if (!nb) continue;
      if (std::find(list.begin(), list.end(), nb) == list.end()) {
        if (!allow_external) return fail(GBCFD_ERR_ARG, "a connected neighbour is missing from the block list");
        list.push_back(nb);
      }
    }
  }
  if ((int)list.size() > MAX_GROUP) return fail(GBCFD_ERR_ARG, "too many blocks in one group");
  G->n = (int)list.size();
  long long total = 0;
  int elem0 = -1;
  for (int i = 0; i < G->n; ++i) {
    gbcfd_block b = list[i];
    HaloBlock& h = G->b[i];
    int elem, nvar;
    field_of(b, field, &h.base[0], &elem, &nvar);
    if (elem0 < 0) elem0 = elem;
    if (elem != elem0) return fail(GBCFD_ERR_ARG, "blocks of one group must share a precision");
    G->elem = elem;
    G->nvar = nvar;
    h.nx = b->nx; h.ny = b->ny; h.nz = b->nz;
    h.pitch = elem == 8 ? b->g.px : b->g.pxf;
    for (int f = 0; f < 6; ++f) {
      h.nbr[f] = -1;
      if (b->nbr[f]) h.nbr[f] = (int)(std::find(list.begin(), list.end(), b->nbr[f]) - list.begin());
    }
    if (i < n) {
      h.first = total;
      total += (long long)(b->nx + 4) * (b->ny + 4) * (b->nz + 4) - (long long)b->nx * b->ny * b->nz;
    } else {
      h.first = 0x7fffffffffffffffLL;  // source only: never selected by the halo search
    }
  }
  G->total = total;
  return GBCFD_OK;
}

// ghost cells of the physical faces of blocks[0..n) for `field` (a stage input), one launch per
// direction that has such faces, x before y before z (edges read the earlier directions' ghosts)
static int apply_bc(const gbcfd_block* blocks, int n, int field, cudaStream_t s) {
  for (int i = 0; i < n; ++i) {
    gbcfd_block b = blocks[i];
    const bool mixed = b->p.precision == GBCFD_MIXED;
    BcBlock B;
    memset(&B, 0, sizeof(B));
    B.g = b->g;
    for (int f = 0; f < 6; ++f) B.kind[f] = b->nbr[f] ? GBCFD_BC_NONE : b->bc_kind[f];
    for (int v = 0; v < 5; ++v) B.inf[v] = b->bc_inf[v];
    B.gamma = b->p.gamma;
    B.metrics = b->curvi ? b->metrics : nullptr;
    if (!mixed) {
      B.mode = BC_F64;
      B.field = field == F_STATE ? b->q[0] : (field == F_STAGE1 ? b->q[1] : b->q[2]);
    } else if (field == F_STATE) {
      B.mode = BC_F32;
      B.field = b->sh[b->cur];
    } else {
      B.mode = BC_F32_INC;
      B.field = field == F_STAGE1 ? b->d[0] : b->d[1];
      B.shadow = b->sh[b->cur];
    }
    for (int d = 0; d < 3; ++d) {
      if (B.kind[2 * d] == GBCFD_BC_NONE && B.kind[2 * d + 1] == GBCFD_BC_NONE) continue;
      B.dim = d;
      CK(launch_bc(B, s));
    }
  }
  return GBCFD_OK;
}

static int exchange(const gbcfd_block* blocks, int n, int field, bool allow_external, cudaStream_t s) {
  static thread_local HaloGroup G;  // ~8 KB, kept off the stack
  int rc = build_group(blocks, n, field, allow_external, &G);
  if (rc) return rc;
  CK(launch_halo(G, s));
  if (field != F_METRICS) return apply_bc(blocks, n, field, s);
  return GBCFD_OK;
}

// metric halos and, for blocks holding a state, the time step evaluated on the full metrics;
// run before anything reads metrics after gbcfd_set_metrics
static int init_rate(gbcfd_block b, cudaStream_t s) {
  if (b->curvi)
    CK(launch_init_rate_curvi(b->g, physics_of(b), state_ptr(b), b->metrics, b->ctrl, b->partial, 4 * b->nsm,
                              b->p.precision == GBCFD_MIXED, b->dtl, s));
  else
    CK(launch_init_rate(b->g, physics_of(b), state_ptr(b), b->ctrl, b->partial, 4 * b->nsm,
                        b->p.precision == GBCFD_MIXED, b->dtl, s));
  return GBCFD_OK;
}

static int prepare_metrics(const gbcfd_block* blocks, int n, cudaStream_t s) {
  bool dirty = false;
  for (int i = 0; i < n; ++i) dirty = dirty || blocks[i]->metrics_dirty;
  if (!dirty) return GBCFD_OK;
  int rc = exchange(blocks, n, F_METRICS, true, s);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    if (!blocks[i]->metrics_dirty) continue;
    blocks[i]->metrics_dirty = 0;
    if (blocks[i]->has_state) {
      rc = init_rate(blocks[i], s);
      if (rc) return rc;
    }
  }
  return GBCFD_OK;
}

static int check_blocks(const gbcfd_block* blocks, int n) {
  if (!blocks || n < 1) return fail(GBCFD_ERR_ARG, "empty block list");
  if (n > MAX_GROUP) return fail(GBCFD_ERR_ARG, "too many blocks in one call");
  for (int i = 0; i < n; ++i) {
    if (!blocks[i]) return fail(GBCFD_ERR_ARG, "NULL block in list");
    if (!blocks[i]->has_state) return fail(GBCFD_ERR_STATE, "block has no state");
    if (blocks[i]->p.precision != blocks[0]->p.precision) return fail(GBCFD_ERR_ARG, "mixed precisions in one call");
    if (blocks[i]->next_stage != blocks[0]->next_stage)
      return fail(GBCFD_ERR_STATE, "blocks of one call are at different Runge-Kutta stages");
  }
  return GBCFD_OK;
}

// the field the next stage reads: Q^n before stage 1, the stage-1 output before stage 2, ...
static int input_field(gbcfd_block b) {
  return b->next_stage == 1 ? F_STATE : (b->next_stage == 2 ? F_STAGE1 : F_STAGE2);
}

extern "C" int gbcfd_exchange_halos(const gbcfd_block* blocks, int n, void* stream) {
  int rc = check_blocks(blocks, n);
  if (rc) return rc;
  rc = prepare_metrics(blocks, n, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return exchange(blocks, n, input_field(blocks[0]), true, static_cast<cudaStream_t>(stream));
}

// ---- stages --------------------------------------------------------------------------------
static int run_stage(gbcfd_block b, int stage, double* rout, cudaStream_t s) {
  GroupParams P;
  memset(&P, 0, sizeof(P));
  P.table = b->desc;
  P.nblocks = 1;
  P.cur = b->cur;
  P.ph = physics_of(b);
  P.pk = path_consts(P.ph);
  P.gctrl = b->ctrl;
  P.partial = b->partial;
  P.rout = rout;
  CK(launch_stage(b->p.precision, b->p.viscous, b->curvi, stage, P, b->grid, s));
  if (stage == 3 && b->p.precision == GBCFD_MIXED) b->cur = 1 - b->cur;
  return GBCFD_OK;
}

extern "C" int gbcfd_stage(const gbcfd_block* blocks, int n, int stage, void* stream) {
  int rc = check_blocks(blocks, n);
  if (rc) return rc;
  if (stage < 1 || stage > 3) return fail(GBCFD_ERR_ARG, "stage must be 1, 2 or 3");
  if (stage != blocks[0]->next_stage)
    return fail(GBCFD_ERR_STATE, "stage " + std::to_string(stage) + " called, stage " +
                                     std::to_string(blocks[0]->next_stage) + " expected");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (stage == 1 && n > 1) {
    std::vector<DevCtrl*> c(n);
    for (int i = 0; i < n; ++i) c[i] = blocks[i]->ctrl;
    CK(launch_group_dt(c.data(), n, blocks[0]->p.cfl, s));
  }
  for (int i = 0; i < n; ++i) {
    rc = run_stage(blocks[i], stage, nullptr, s);
    if (rc) return rc;
  }
  if (stage == 3 && n > 1) {  // every block then holds the global step the next stage 1 takes
    std::vector<DevCtrl*> c(n);
    for (int i = 0; i < n; ++i) c[i] = blocks[i]->ctrl;
    CK(launch_group_dt(c.data(), n, blocks[0]->p.cfl, s));
  }
  for (int i = 0; i < n; ++i) blocks[i]->next_stage = stage % 3 + 1;
  return GBCFD_OK;
}

extern "C" int gbcfd_step(const gbcfd_block* blocks, int n, int nsteps, void* stream) {
  int rc = check_blocks(blocks, n);
  if (rc) return rc;
  if (nsteps < 0) return fail(GBCFD_ERR_ARG, "nsteps must be >= 0");
  if (blocks[0]->next_stage != 1) return fail(GBCFD_ERR_STATE, "a step was left between stages");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = prepare_metrics(blocks, n, s);
  if (rc) return rc;
  const int fields[3] = {F_STATE, F_STAGE1, F_STAGE2};
  for (int it = 0; it < nsteps; ++it) {
    for (int st = 1; st <= 3; ++st) {
      rc = exchange(blocks, n, fields[st - 1], false, s);
      if (rc) return rc;
      rc = gbcfd_stage(blocks, n, st, stream);
      if (rc) return rc;
    }
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_compute_residual(gbcfd_block b, double* r, void* stream) {
  if (!b || !r) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (!b->has_state) return fail(GBCFD_ERR_STATE, "no state set");
  bool dev = false;
  int rc = is_device_ptr(r, &dev);
  if (rc) return rc;
  if (!dev) return fail(GBCFD_ERR_ARG, "r must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = prepare_metrics(&b, 1, s);
  if (rc) return rc;
  rc = exchange(&b, 1, F_STATE, true, s);
  if (rc) return rc;
  return run_stage(b, 0, r, s);
}

// ---- batched groups ------------------------------------------------------------------------
struct gbcfd_group_s {
  std::vector<gbcfd_block> blocks;
  std::vector<BlockDesc> table_host;
  BlockDesc* table;
  DevCtrl* gctrl;
  double* partial;
  size_t partial_n;
  int ctas_per_sm;        // grid = SMs x this (split between the blocks)
  int ty;                 // tile height of the stage kernel the table is written for
  int push_ok;            // the members form a conforming lattice (group_can_push)
  int push;               // stages 1 and 2 fill the neighbours' halos themselves (a schedule choice)
  int grid;
  cudaStream_t cap;       // private stream the step graphs are captured on
  cudaGraphExec_t exec[2];  // one step, for each parity of the mixed path's ping-pong
  cudaEvent_t marks[7];     // caller's timing events (or none)
  bool timed;
  std::vector<unsigned> versions;  // members' descriptor versions the table was written with
};

static int max_group_ctas(int nsm) { return 16 * nsm; }

extern "C" int gbcfd_group_required_bytes(int n, size_t* bytes) {
  if (n < 1 || n > MAX_GROUP) return fail(GBCFD_ERR_ARG, "a group holds 1.." + std::to_string(MAX_GROUP) + " blocks");
  if (!bytes) return fail(GBCFD_ERR_ARG, "bytes is NULL");
  int dev = 0, nsm = 0;
  int rc = device_sms(&dev, &nsm);
  if (rc) return rc;
  *bytes = align256(sizeof(BlockDesc) * n) + align256(sizeof(DevCtrl)) +
           align256(sizeof(double) * NPART * (size_t)(max_group_ctas(nsm) + n));
  return GBCFD_OK;
}

// the members' face neighbours as group indices, in every descriptor of the table
static void set_group_nbrs(gbcfd_group g) {
  for (size_t i = 0; i < g->blocks.size(); ++i)
    for (int f = 0; f < 6; ++f) {
      gbcfd_block nb = g->blocks[i]->nbr[f];
      g->table_host[i].nbr[f] = nb ? (int)(std::find(g->blocks.begin(), g->blocks.end(), nb) - g->blocks.begin()) : -1;
    }
}

// Whether the stage kernel may fill the halos itself (push_halo in stage.cuh): Cartesian Euler
// blocks (the kernels compiled with the fold) forming a conforming block lattice -- every face connected to a member (periodic wrap included), the two
// blocks of a face equal in the face's two directions, at least HALO cells in every direction,
// and walking face neighbours along two different axes reaching the same block in either order --
// so each halo cell has exactly one source cell, the one the halo kernel would copy.
static bool group_can_push(const std::vector<gbcfd_block>& bl) {
  auto nb = [](gbcfd_block b, int f) { return b ? b->nbr[f] : nullptr; };
  if (bl[0]->p.viscous || bl[0]->curvi) return false;  // the folded kernels: Cartesian Euler blocks
  for (gbcfd_block b : bl) {
    if (b->nx < HALO || b->ny < HALO || b->nz < HALO) return false;
    for (int f = 0; f < 6; ++f) {
      gbcfd_block n = b->nbr[f];
      if (!n || n->nbr[f ^ 1] != b) return false;
      const int a = f >> 1;  // axis of the face: the other two sizes must match
      if ((a != 0 && n->nx != b->nx) || (a != 1 && n->ny != b->ny) || (a != 2 && n->nz != b->nz)) return false;
    }
    for (int f1 = 0; f1 < 6; ++f1)
      for (int f2 = 0; f2 < 6; ++f2)
        if ((f1 >> 1) != (f2 >> 1) && nb(nb(b, f1), f2) != nb(nb(b, f2), f1)) return false;
  }
  return true;
}

// split SMs x ctas_per_sm CTAs between the blocks in proportion to their tile-planes (each gets
// at least one) and write the descriptor table for the stage kernel of tile height ty
static int group_split(gbcfd_group g, int ctas_per_sm, cudaStream_t s, int ty = -1) {
  const int nsm = g->blocks[0]->nsm;
  if (ty < 0) ty = g->ty;
  g->versions.resize(g->blocks.size());
  for (size_t i = 0; i < g->blocks.size(); ++i) {  // the members' current descriptors
    int rc = write_desc(g->blocks[i], ty, &g->table_host[i]);
    if (rc) return rc;
    g->versions[i] = g->blocks[i]->desc_version;
  }
  set_group_nbrs(g);
  const long long target = (long long)nsm * ctas_per_sm;
  long long W = 0;
  for (auto& d : g->table_host) W += d.units;
  int c0 = 0;
  for (size_t i = 0; i < g->table_host.size(); ++i) {
    BlockDesc& d = g->table_host[i];
    long long c = (target * d.units + W / 2) / W;
    c = std::max(1LL, std::min(c, d.units));
    d.cta0 = c0;
    d.ctas = (int)c;
    c0 += (int)c;
  }
  if ((size_t)c0 > g->partial_n) return fail(GBCFD_ERR_ARG, "too many CTAs for the group's partial sums");
  g->grid = c0;
  g->ctas_per_sm = ctas_per_sm;
  g->ty = ty;
  CK(cudaMemcpyAsync(g->table, g->table_host.data(), sizeof(BlockDesc) * g->table_host.size(),
                     cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host table is reused
  for (int p = 0; p < 2; ++p)
    if (g->exec[p]) { cudaGraphExecDestroy(g->exec[p]); g->exec[p] = nullptr; }
  return GBCFD_OK;
}

extern "C" int gbcfd_group_create(const gbcfd_block* blocks, int n, void* dev_mem, size_t bytes, gbcfd_group* out) {
  if (!out) return fail(GBCFD_ERR_ARG, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  int rc = gbcfd_group_required_bytes(n, &need);
  if (rc) return rc;
  if (!blocks || !dev_mem) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (((uintptr_t)dev_mem & 255u) != 0) return fail(GBCFD_ERR_MEMORY, "dev_mem must be 256-byte aligned");
  if (bytes < need) return fail(GBCFD_ERR_MEMORY, "dev_mem smaller than gbcfd_group_required_bytes");
  for (int i = 0; i < n; ++i) {
    gbcfd_block b = blocks[i];
    if (!b) return fail(GBCFD_ERR_ARG, "NULL block");
    const gbcfd_params &p = b->p, &q = blocks[0]->p;
    if (p.precision != q.precision || p.viscous != q.viscous || p.limiter != q.limiter || p.gamma != q.gamma ||
        p.local_dt != q.local_dt ||
        p.mu != q.mu || p.Pr != q.Pr || p.cfl != q.cfl || p.entropy_eps != q.entropy_eps ||
        b->curvi != blocks[0]->curvi)
      return fail(GBCFD_ERR_ARG, "group members must share precision, physics and grid kind");
    for (int j = 0; j < i; ++j)
      if (blocks[j] == b) return fail(GBCFD_ERR_ARG, "a block appears twice in the group");
    for (int f = 0; f < 6; ++f)
      if (b->nbr[f] && std::find(blocks, blocks + n, b->nbr[f]) == blocks + n)
        return fail(GBCFD_ERR_ARG, "a connected neighbour is not a member of the group");
  }
  gbcfd_group g = new gbcfd_group_s();
  g->blocks.assign(blocks, blocks + n);
  char* base = static_cast<char*>(dev_mem);
  g->table = reinterpret_cast<BlockDesc*>(base);
  g->gctrl = reinterpret_cast<DevCtrl*>(base + align256(sizeof(BlockDesc) * n));
  g->partial = reinterpret_cast<double*>(base + align256(sizeof(BlockDesc) * n) + align256(sizeof(DevCtrl)));
  g->partial_n = (size_t)max_group_ctas(blocks[0]->nsm) + n;
  g->exec[0] = g->exec[1] = nullptr;
  g->cap = nullptr;
  g->timed = false;
  g->ty = TY_DEFAULT;
  g->push_ok = group_can_push(g->blocks) ? 1 : 0;
  g->push = 0;
  for (int i = 0; i < n; ++i) g->table_host.push_back(blocks[i]->desc_host);
  const int mixed = blocks[0]->p.precision == GBCFD_MIXED, vis = blocks[0]->p.viscous, cv = blocks[0]->curvi;
  cudaError_t e = mixed ? (cv ? stage_prepare_f32c(vis) : stage_prepare_f32(vis))
                        : (cv ? stage_prepare_f64c(vis) : stage_prepare_f64(vis));
  if (e == cudaSuccess) e = cudaMemset(g->gctrl, 0, sizeof(DevCtrl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete g; return cuda_fail(e, "group set-up"); }
  const int occ = blocks[0]->p.precision == GBCFD_MIXED
                      ? (blocks[0]->curvi ? stage_occupancy_f32c(blocks[0]->p.viscous) : stage_occupancy_f32(blocks[0]->p.viscous))
                      : (blocks[0]->curvi ? stage_occupancy_f64c(blocks[0]->p.viscous) : stage_occupancy_f64(blocks[0]->p.viscous));
  rc = group_split(g, occ, g->cap, TY_DEFAULT);
  if (rc) { cudaStreamDestroy(g->cap); delete g; return rc; }
  *out = g;
  return GBCFD_OK;
}

extern "C" int gbcfd_group_destroy(gbcfd_group g) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  for (int p = 0; p < 2; ++p)
    if (g->exec[p]) cudaGraphExecDestroy(g->exec[p]);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  return GBCFD_OK;
}

static GroupParams group_params(gbcfd_group g) {
  GroupParams P;
  memset(&P, 0, sizeof(P));
  P.table = g->table;
  P.nblocks = (int)g->blocks.size();
  P.cur = g->blocks[0]->cur;
  P.ph = physics_of(g->blocks[0]);
  P.pk = path_consts(P.ph);
  P.gctrl = g->gctrl;
  P.partial = g->partial;
  P.push = g->push;
  return P;
}

// one step of the group enqueued on s: time step, then halo exchange and one batched stage
// launch, three times
static int group_step_launches(gbcfd_group g, cudaStream_t s) {
  const int n = (int)g->blocks.size();
  gbcfd_block b0 = g->blocks[0];
  std::vector<DevCtrl*> ctrls(n);
  for (int i = 0; i < n; ++i) ctrls[i] = g->blocks[i]->ctrl;
  auto mark = [&](int i) { return g->timed ? cudaEventRecordWithFlags(g->marks[i], s, cudaEventRecordExternal)
                                            : cudaSuccess; };
  CK(mark(0));
  CK(launch_group_dt(ctrls.data(), n, b0->p.cfl, s, g->gctrl));
  GroupParams P = group_params(g);
  const int fields[3] = {F_STATE, F_STAGE1, F_STAGE2};
  for (int st = 1; st <= 3; ++st) {
    if (st == 1 || !g->push) {  // with push, stages 1 and 2 fill the halos stages 2 and 3 read
      int rc = exchange(g->blocks.data(), n, fields[st - 1], false, s);
      if (rc) return rc;
    }
    CK(mark(2 * st - 1));
    CK(launch_stage(b0->p.precision, b0->p.viscous, b0->curvi, st, P, g->grid, s, g->ty));
    CK(mark(2 * st));
  }
  return GBCFD_OK;
}

static int group_check(gbcfd_group g) {
  int rc = check_blocks(g->blocks.data(), (int)g->blocks.size());
  if (rc) return rc;
  for (auto b : g->blocks) {
    if (b->next_stage != 1) return fail(GBCFD_ERR_STATE, "a group member was left between stages");
    if (b->cur != g->blocks[0]->cur) return fail(GBCFD_ERR_STATE, "group members are at different step parities");
  }
  return GBCFD_OK;
}

// rewrite the table when a member's descriptor changed (the graphs read it from device memory)
static int group_refresh(gbcfd_group g, cudaStream_t s) {
  bool changed = false;
  for (size_t i = 0; i < g->blocks.size(); ++i) changed = changed || g->versions[i] != g->blocks[i]->desc_version;
  if (!changed) return GBCFD_OK;
  for (size_t i = 0; i < g->blocks.size(); ++i) {
    const int cta0 = g->table_host[i].cta0, ctas = g->table_host[i].ctas;
    int rc = write_desc(g->blocks[i], g->ty, &g->table_host[i]);
    if (rc) return rc;
    g->table_host[i].cta0 = cta0;
    g->table_host[i].ctas = ctas;
    g->versions[i] = g->blocks[i]->desc_version;
  }
  set_group_nbrs(g);
  CK(cudaMemcpyAsync(g->table, g->table_host.data(), sizeof(BlockDesc) * g->table_host.size(),
                     cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host table is reused
  return GBCFD_OK;
}

extern "C" int gbcfd_group_step(gbcfd_group g, int nsteps, void* stream) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  if (nsteps < 0) return fail(GBCFD_ERR_ARG, "nsteps must be >= 0");
  int rc = group_check(g);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = group_refresh(g, s);
  if (rc) return rc;
  rc = prepare_metrics(g->blocks.data(), (int)g->blocks.size(), s);
  if (rc) return rc;
  const bool mixed = g->blocks[0]->p.precision == GBCFD_MIXED;
  for (int it = 0; it < nsteps; ++it) {
    const int par = mixed ? g->blocks[0]->cur : 0;
    if (!g->exec[par]) {  // capture one step on the private stream
      CK(cudaStreamSynchronize(s));
      CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
      rc = group_step_launches(g, g->cap);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
      if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&g->exec[par], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(g->exec[par], s));
    if (mixed)
      for (auto b : g->blocks) b->cur = 1 - b->cur;
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_group_set_timing(gbcfd_group g, void* const* events, int n) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  if (events && n != 7) return fail(GBCFD_ERR_ARG, "timing needs exactly 7 events");
  if (events)
    for (int i = 0; i < 7; ++i)
      if (!events[i]) return fail(GBCFD_ERR_ARG, "NULL event");
  g->timed = events != nullptr;
  for (int i = 0; i < 7; ++i) g->marks[i] = events ? static_cast<cudaEvent_t>(events[i]) : nullptr;
  for (int p = 0; p < 2; ++p)
    if (g->exec[p]) { cudaGraphExecDestroy(g->exec[p]); g->exec[p] = nullptr; }
  return GBCFD_OK;
}

extern "C" int gbcfd_group_set_schedule(gbcfd_group g, int ctas_per_sm, int tile_rows, int halo_push,
                                        void* stream) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  gbcfd_block b0 = g->blocks[0];
  int tys[4];
  const int ntile = stage_tiles(b0->p.precision, b0->p.viscous, b0->curvi, tys);
  if (std::find(tys, tys + ntile, tile_rows) == tys + ntile)
    return fail(GBCFD_ERR_ARG, "tile height " + std::to_string(tile_rows) + " is not compiled for this path");
  if (ctas_per_sm < 1 || (long long)b0->nsm * ctas_per_sm > max_group_ctas(b0->nsm))
    return fail(GBCFD_ERR_ARG, "ctas_per_sm must be 1..16");
  if (halo_push && !g->push_ok)
    return fail(GBCFD_ERR_ARG, "halo push needs a conforming periodic block lattice (every face connected, "
                               "matching face sizes, at least 2 cells per direction)");
  if (stage_prepare_tile(b0->p.precision, b0->p.viscous, b0->curvi, tile_rows) != cudaSuccess ||
      (halo_push && (b0->p.precision == GBCFD_MIXED ? stage_prepare_f32_push(tile_rows)
                                                    : stage_prepare_f64_push(tile_rows)) != cudaSuccess))
    return fail(GBCFD_ERR_CUDA, "stage kernel set-up failed");
  g->push = halo_push ? 1 : 0;
  return group_split(g, ctas_per_sm, static_cast<cudaStream_t>(stream), tile_rows);
}

extern "C" int gbcfd_group_get_schedule(gbcfd_group g, int* ctas_per_sm, int* tile_rows, int* halo_push) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  if (ctas_per_sm) *ctas_per_sm = g->ctas_per_sm;
  if (tile_rows) *tile_rows = g->ty;
  if (halo_push) *halo_push = g->push;
  return GBCFD_OK;
}

extern "C" int gbcfd_group_tune(gbcfd_group g, void* stream, int* ctas_per_sm) {
  return gbcfd_group_tune_tile(g, stream, ctas_per_sm, nullptr);
}

extern "C" int gbcfd_group_tune_tile(gbcfd_group g, void* stream, int* ctas_per_sm, int* tile_rows) {
  if (!g) return fail(GBCFD_ERR_ARG, "group is NULL");
  int rc = group_check(g);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = prepare_metrics(g->blocks.data(), (int)g->blocks.size(), s);
  if (rc) return rc;
  gbcfd_block b0 = g->blocks[0];
  // candidates: every tile height compiled for the path, each with one resident wave (occ CTAs
  // per SM) and finer splits of 2x .. 16x that, up to 16 CTAs per SM: uneven blocks share the
  // grid in proportion to their tile-planes with rounding, and several waves of smaller CTAs
  // even that out (on the 96-block lattice 8 per SM beat 1 by 30% on the FP64 path)
  int tys[4];
  const int ntile = stage_tiles(b0->p.precision, b0->p.viscous, b0->curvi, tys);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_c = 0, best_ty = TY_DEFAULT;
  rc = exchange(g->blocks.data(), (int)g->blocks.size(), F_STATE, false, s);
  g->push = 0;  // shapes are compared with the exchange as a launch; the fold is decided after
  for (int ti = 0; ti < ntile && !rc; ++ti) {
    const int ty = tys[ti];
    if (stage_prepare_tile(b0->p.precision, b0->p.viscous, b0->curvi, ty) != cudaSuccess) {
      rc = fail(GBCFD_ERR_CUDA, "stage kernel set-up failed");
      break;
    }
    const int occ = stage_occupancy_tile(b0->p.precision, b0->p.viscous, b0->curvi, ty);
    const int cand[5] = {occ, 2 * occ, 4 * occ, 8 * occ, 16 * occ};
    for (int ci = 0; ci < 5 && !rc; ++ci) {
      if ((long long)b0->nsm * cand[ci] > max_group_ctas(b0->nsm)) continue;
      rc = group_split(g, cand[ci], s, ty);
      if (rc) break;
      GroupParams P = group_params(g);
      float t = 0.f;
      // stages 1 and 2 write only the stage scratch (Q1 / Q2, or D1 / D2) and the norms, so they
      // can run without touching the state; stage 2 reads stage 1's output with its halos
      for (int rep = 0; rep < 3 && !rc; ++rep) {  // the first pair warms up, two are timed
        float ms1 = 0.f, ms2 = 0.f;
        cudaEventRecord(e0, s);
        if (launch_stage(b0->p.precision, b0->p.viscous, b0->curvi, 1, P, g->grid, s, ty) != cudaSuccess)
          rc = fail(GBCFD_ERR_CUDA, "tuning launch failed");
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms1, e0, e1);
        if (!rc) rc = exchange(g->blocks.data(), (int)g->blocks.size(), F_STAGE1, false, s);
        if (rc) break;
        cudaEventRecord(e0, s);
        if (launch_stage(b0->p.precision, b0->p.viscous, b0->curvi, 2, P, g->grid, s, ty) != cudaSuccess)
          rc = fail(GBCFD_ERR_CUDA, "tuning launch failed");
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms2, e0, e1);
        if (rep > 0) t += ms1 + ms2;
      }
      if (!rc && t < best) { best = t; best_c = cand[ci]; best_ty = ty; }
    }
  }
  // the halo exchange of the stage output: a launch between the stages, or folded into the
  // stages (push); timed on the chosen shape as stage 1, [exchange,] stage 2
  g->push = 0;
  if (!rc) rc = group_split(g, best_c, s, best_ty);
  if (!rc && g->push_ok &&
      (b0->p.precision == GBCFD_MIXED ? stage_prepare_f32_push(best_ty) : stage_prepare_f64_push(best_ty)) !=
          cudaSuccess)
    rc = fail(GBCFD_ERR_CUDA, "stage kernel set-up failed");
  if (!rc && g->push_ok) {
    float tp[2] = {0.f, 0.f};
    for (int push = 0; push < 2 && !rc; ++push) {
      g->push = push;
      GroupParams P = group_params(g);
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, s);
        if (launch_stage(b0->p.precision, b0->p.viscous, b0->curvi, 1, P, g->grid, s, best_ty) != cudaSuccess)
          rc = fail(GBCFD_ERR_CUDA, "tuning launch failed");
        if (!rc && !push) rc = exchange(g->blocks.data(), (int)g->blocks.size(), F_STAGE1, false, s);
        if (!rc && launch_stage(b0->p.precision, b0->p.viscous, b0->curvi, 2, P, g->grid, s, best_ty) != cudaSuccess)
          rc = fail(GBCFD_ERR_CUDA, "tuning launch failed");
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tp[push] += ms;
      }
    }
    g->push = (!rc && tp[1] < tp[0]) ? 1 : 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) { g->push = 0; return rc; }
  for (int p = 0; p < 2; ++p)  // the step graphs hold the exchange choice
    if (g->exec[p]) { cudaGraphExecDestroy(g->exec[p]); g->exec[p] = nullptr; }
  if (ctas_per_sm) *ctas_per_sm = best_c;
  if (tile_rows) *tile_rows = best_ty;
  return GBCFD_OK;
}

// ---- read-backs ----------------------------------------------------------------------------
static int read_ctrl(gbcfd_block b, DevCtrl* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h, b->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GBCFD_OK;
}

extern "C" int gbcfd_residual_norm(gbcfd_block b, double out[5], void* stream) {
  if (!b || !out) return fail(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevCtrl h;
  int rc = read_ctrl(b, &h, s);
  if (rc) return rc;
  for (int m = 0; m < 5; ++m) out[m] = h.norms[m];
  if (h.flag) {
    CK(cudaMemsetAsync(&b->ctrl->flag, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    if (h.flag & FLAG_TIMEOUT) return fail(GBCFD_ERR_TIMEOUT, "a bounded device wait timed out");
    return fail(GBCFD_ERR_NONPHYSICAL, "non-positive density or pressure, or a non-finite value");
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_get_dt(gbcfd_block b, double* dt, void* stream) {
  if (!b || !dt) return fail(GBCFD_ERR_ARG, "NULL argument");
  DevCtrl h;
  int rc = read_ctrl(b, &h, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  *dt = h.dt;
  return GBCFD_OK;
}

// ---- host-to-host pipeline ----------------------------------------------------------------
// Items (a host state, nsteps steps, the host result) rotate over the members.  Three streams
// carry the uploads (copy engine, host -> the member's landing area), the device work (state
// from the landing area, the steps, the result back into it) and the downloads (copy engine,
// landing area -> host).  Item i+1's upload and item i-1's download use the two directions of
// the host link while item i steps; a member takes its next item only after the download of its
// previous one (events).
struct gbcfd_pipe_s {
  std::vector<PipeMember> members;
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  std::vector<cudaEvent_t> up_done, comp_done, down_done;  // per member, of its latest item
  long long items = 0;
  int broken = 0;  // an item failed after its upload was enqueued: no new items until a sync
};

static void pipe_release(gbcfd_pipe p) {
  if (p->up) cudaStreamSynchronize(p->up);
  if (p->comp) cudaStreamSynchronize(p->comp);
  if (p->down) cudaStreamSynchronize(p->down);
  for (auto* v : {&p->up_done, &p->comp_done, &p->down_done})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  for (cudaStream_t s : {p->up, p->comp, p->down})
    if (s) cudaStreamDestroy(s);
  for (const PipeMember& m : p->members)
    if (m.release) m.release(m.self);
  delete p;
}

static bool page_locked(const void* ptr) {
  bool dev = false;
  void* mapped = nullptr;
  if (locate_ptr(ptr, &dev, &mapped) != GBCFD_OK) return false;
  return !dev && mapped != nullptr;
}

// takes ownership of the members (released with the pipeline, or here when creation fails)
int gbcfd::pipe_create(const PipeMember* members, int n, gbcfd_pipe* out) {
  gbcfd_pipe p = new gbcfd_pipe_s;
  p->members.assign(members, members + n);
  p->up_done.assign(n, nullptr);
  p->comp_done.assign(n, nullptr);
  p->down_done.assign(n, nullptr);
  cudaError_t e = cudaDeviceSynchronize();  // the members' earlier work (any stream) is done
  for (cudaStream_t* s : {&p->up, &p->comp, &p->down})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  for (auto* v : {&p->up_done, &p->comp_done, &p->down_done})
    for (cudaEvent_t& ev : *v)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    pipe_release(p);
    return cuda_fail(e, "pipeline streams and events");
  }
  *out = p;
  return GBCFD_OK;
}

// finite-volume members: the landing area is the block's staging area
static int fv_upload(void* self, const double* q_in, cudaStream_t s) {
  gbcfd_block b = static_cast<gbcfd_block>(self);
  CK(cudaMemcpyAsync(b->staging, q_in, sizeof(double) * 5 * (size_t)b->nx * b->ny * b->nz,
                     cudaMemcpyHostToDevice, s));
  return GBCFD_OK;
}
static int fv_run(void* self, int nsteps, cudaStream_t s) {
  gbcfd_block b = static_cast<gbcfd_block>(self);
  if (b->next_stage != 1) return fail(GBCFD_ERR_STATE, "a member block was left between stages");
  // the state as gbcfd_set_state sets it from device memory
  CK(launch_scatter(b->g, reinterpret_cast<const double*>(b->staging), state_ptr(b),
                    b->p.precision == GBCFD_MIXED ? b->sh[b->cur] : nullptr, s));
  b->has_state = 1;
  b->next_stage = 1;
  int rc = b->metrics_dirty ? prepare_metrics(&b, 1, s) : init_rate(b, s);
  if (rc) return rc;
  rc = gbcfd_step(&b, 1, nsteps, s);
  if (rc) return rc;
  CK(launch_gather(b->g, state_ptr(b), reinterpret_cast<double*>(b->staging), s));
  return GBCFD_OK;
}
static int fv_download(void* self, double* q_out, double* norms, int nsteps, cudaStream_t s) {
  gbcfd_block b = static_cast<gbcfd_block>(self);
  CK(cudaMemcpyAsync(q_out, b->staging, sizeof(double) * 5 * (size_t)b->nx * b->ny * b->nz,
                     cudaMemcpyDeviceToHost, s));
  if (norms && nsteps > 0) CK(cudaMemcpyAsync(norms, b->ctrl->norms, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return GBCFD_OK;
}
static int fv_flags(void* self, cudaStream_t s, int* flags) {
  gbcfd_block b = static_cast<gbcfd_block>(self);
  DevCtrl h;
  const int rc = read_ctrl(b, &h, s);
  if (rc) return rc;
  *flags = h.flag;
  if (h.flag) {
    CK(cudaMemsetAsync(&b->ctrl->flag, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_pipe_create(const gbcfd_block* blocks, int n, gbcfd_pipe* out) {
  if (!blocks || !out) return fail(GBCFD_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > 8) return fail(GBCFD_ERR_ARG, "a pipeline takes 1 to 8 blocks");
  const gbcfd_block a = blocks[0];
  if (!a) return fail(GBCFD_ERR_ARG, "NULL block");
  const size_t bytes = sizeof(double) * 5 * (size_t)a->nx * a->ny * a->nz;
  std::vector<PipeMember> m(n);
  for (int i = 0; i < n; ++i) {
    const gbcfd_block b = blocks[i];
    if (!b) return fail(GBCFD_ERR_ARG, "NULL block");
    for (int k = 0; k < i; ++k)
      if (blocks[k] == b) return fail(GBCFD_ERR_ARG, "a block is listed twice");
    if (b->nx != a->nx || b->ny != a->ny || b->nz != a->nz) return fail(GBCFD_ERR_ARG, "members differ in size");
    if (memcmp(&b->p, &a->p, sizeof(gbcfd_params)) != 0) return fail(GBCFD_ERR_ARG, "members differ in parameters");
    if (b->curvi != a->curvi || memcmp(b->spacing, a->spacing, sizeof(a->spacing)) != 0)
      return fail(GBCFD_ERR_ARG, "members differ in grid");
    for (int f = 0; f < 6; ++f) {
      if (b->nbr[f] && b->nbr[f] != b) return fail(GBCFD_ERR_ARG, "members must not connect to other blocks");
      if (!b->nbr[f] != !a->nbr[f] || (!b->nbr[f] && b->bc_kind[f] != a->bc_kind[f]))
        return fail(GBCFD_ERR_ARG, "members differ in boundary conditions");
    }
    if (b->staging_bytes < bytes) return fail(GBCFD_ERR_MEMORY, "member staging area too small");
    m[i] = PipeMember{b, bytes, fv_upload, fv_run, fv_download, fv_flags, nullptr};
  }
  return pipe_create(m.data(), n, out);
}

// group members: an item is the concatenation of the member blocks' compact states, in the
// group's block order; each block lands in its own staging area
struct GroupMember {
  gbcfd_group g;
  std::vector<size_t> off;  // byte offset of each block's state in the item
  size_t bytes;
};
static size_t compact_bytes(gbcfd_block b) { return sizeof(double) * 5 * (size_t)b->nx * b->ny * b->nz; }
static int gp_upload(void* self, const double* q_in, cudaStream_t s) {
  const GroupMember* G = static_cast<const GroupMember*>(self);
  const char* src = reinterpret_cast<const char*>(q_in);
  for (size_t i = 0; i < G->g->blocks.size(); ++i) {
    gbcfd_block b = G->g->blocks[i];
    CK(cudaMemcpyAsync(b->staging, src + G->off[i], compact_bytes(b), cudaMemcpyHostToDevice, s));
  }
  return GBCFD_OK;
}
static int gp_run(void* self, int nsteps, cudaStream_t s) {
  const GroupMember* G = static_cast<const GroupMember*>(self);
  for (gbcfd_block b : G->g->blocks) {
    if (b->next_stage != 1) return fail(GBCFD_ERR_STATE, "a member block was left between stages");
    CK(launch_scatter(b->g, reinterpret_cast<const double*>(b->staging), state_ptr(b),
                      b->p.precision == GBCFD_MIXED ? b->sh[b->cur] : nullptr, s));
    b->has_state = 1;
    b->next_stage = 1;
    const int rc = b->metrics_dirty ? prepare_metrics(&b, 1, s) : init_rate(b, s);
    if (rc) return rc;
  }
  const int rc = gbcfd_group_step(G->g, nsteps, s);
  if (rc) return rc;
  for (gbcfd_block b : G->g->blocks)
    CK(launch_gather(b->g, state_ptr(b), reinterpret_cast<double*>(b->staging), s));
  return GBCFD_OK;
}
static int gp_download(void* self, double* q_out, double* norms, int nsteps, cudaStream_t s) {
  const GroupMember* G = static_cast<const GroupMember*>(self);
  char* dst = reinterpret_cast<char*>(q_out);
  for (size_t i = 0; i < G->g->blocks.size(); ++i) {
    gbcfd_block b = G->g->blocks[i];
    CK(cudaMemcpyAsync(dst + G->off[i], b->staging, compact_bytes(b), cudaMemcpyDeviceToHost, s));
    if (norms && nsteps > 0)
      CK(cudaMemcpyAsync(norms + 5 * i, b->ctrl->norms, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  return GBCFD_OK;
}
static int gp_flags(void* self, cudaStream_t s, int* flags) {
  const GroupMember* G = static_cast<const GroupMember*>(self);
  *flags = 0;
  for (gbcfd_block b : G->g->blocks) {
    int f = 0;
    const int rc = fv_flags(b, s, &f);
    if (rc) return rc;
    *flags |= f;
  }
  return GBCFD_OK;
}
static void gp_release(void* self) { delete static_cast<GroupMember*>(self); }

extern "C" int gbcfd_group_pipe_create(const gbcfd_group* groups, int n, gbcfd_pipe* out) {
  if (!groups || !out) return fail(GBCFD_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > 8) return fail(GBCFD_ERR_ARG, "a pipeline takes 1 to 8 groups");
  const gbcfd_group a = groups[0];
  if (!a) return fail(GBCFD_ERR_ARG, "NULL group");
  const size_t nb = a->blocks.size();
  std::vector<gbcfd_block> seen;
  for (int i = 0; i < n; ++i) {
    const gbcfd_group g = groups[i];
    if (!g) return fail(GBCFD_ERR_ARG, "NULL group");
    if (g->blocks.size() != nb) return fail(GBCFD_ERR_ARG, "member groups differ in their blocks");
    for (size_t k = 0; k < nb; ++k) {
      const gbcfd_block b = g->blocks[k], r = a->blocks[k];
      if (std::find(seen.begin(), seen.end(), b) != seen.end())
        return fail(GBCFD_ERR_ARG, "a block belongs to two member groups (or a group is listed twice)");
      seen.push_back(b);
      if (b->nx != r->nx || b->ny != r->ny || b->nz != r->nz || memcmp(&b->p, &r->p, sizeof(gbcfd_params)) != 0 ||
          b->curvi != r->curvi || memcmp(b->spacing, r->spacing, sizeof(r->spacing)) != 0)
        return fail(GBCFD_ERR_ARG, "member groups differ in their blocks");
      for (int f = 0; f < 6; ++f) {
        // the same connection pattern: neighbour k' of block k in every group
        const auto idx = [](gbcfd_group G, gbcfd_block x) -> long {
          if (!x) return -1;
          return (long)(std::find(G->blocks.begin(), G->blocks.end(), x) - G->blocks.begin());
        };
        if (idx(g, b->nbr[f]) != idx(a, r->nbr[f]) || (!b->nbr[f] && b->bc_kind[f] != r->bc_kind[f]))
          return fail(GBCFD_ERR_ARG, "member groups differ in connections or boundary conditions");
      }
      if (b->staging_bytes < compact_bytes(b)) return fail(GBCFD_ERR_MEMORY, "member staging area too small");
    }
  }
  std::vector<PipeMember> m(n);
  for (int i = 0; i < n; ++i) {
    GroupMember* G = new GroupMember;
    G->g = groups[i];
    size_t off = 0;
    for (gbcfd_block b : G->g->blocks) {
      G->off.push_back(off);
      off += compact_bytes(b);
    }
    G->bytes = off;
    m[i] = PipeMember{G, off, gp_upload, gp_run, gp_download, gp_flags, gp_release};
  }
  return pipe_create(m.data(), n, out);
}

extern "C" int gbcfd_pipe_destroy(gbcfd_pipe p) {
  if (!p) return fail(GBCFD_ERR_ARG, "NULL pipeline");
  pipe_release(p);
  return GBCFD_OK;
}

extern "C" int gbcfd_pipe_submit(gbcfd_pipe p, const double* q_in, double* q_out, int nsteps, double* norms) {
  if (!p || !q_in || !q_out) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (nsteps < 0) return fail(GBCFD_ERR_ARG, "nsteps must be >= 0");
  if (!page_locked(q_in) || !page_locked(q_out) || (norms && !page_locked(norms)))
    return fail(GBCFD_ERR_ARG, "pipeline buffers must be page-locked host memory");
  if (p->broken) return fail(GBCFD_ERR_STATE, "a pipeline item failed; call gbcfd_pipe_sync first");
  const int nb = (int)p->members.size();
  const int j = (int)(p->items % nb);
  const PipeMember& m = p->members[j];
  // upload: the member's landing area is free once its previous item is downloaded
  if (p->items >= nb) CK(cudaStreamWaitEvent(p->up, p->down_done[j], 0));
  int rc = m.upload(m.self, q_in, p->up);
  if (rc) return rc;
  // from here on a failure leaves work of this item in flight: refuse new items until a sync
  p->broken = 1;
  CK(cudaEventRecord(p->up_done[j], p->up));
  CK(cudaStreamWaitEvent(p->comp, p->up_done[j], 0));
  rc = m.run(m.self, nsteps, p->comp);
  if (rc) return rc;
  CK(cudaEventRecord(p->comp_done[j], p->comp));
  CK(cudaStreamWaitEvent(p->down, p->comp_done[j], 0));
  rc = m.download(m.self, q_out, norms, nsteps, p->down);
  if (rc) return rc;
  CK(cudaEventRecord(p->down_done[j], p->down));
  p->broken = 0;
  p->items++;
  return GBCFD_OK;
}

extern "C" int gbcfd_pipe_sync(gbcfd_pipe p) {
  if (!p) return fail(GBCFD_ERR_ARG, "NULL pipeline");
  CK(cudaStreamSynchronize(p->up));
  CK(cudaStreamSynchronize(p->comp));
  CK(cudaStreamSynchronize(p->down));
  p->broken = 0;  // nothing of a failed item is in flight any more
  int flags = 0;
  for (const PipeMember& m : p->members) {
    int f = 0;
    const int rc = m.flags(m.self, p->comp, &f);
    if (rc) return rc;
    flags |= f;
  }
  if (flags & FLAG_TIMEOUT) return fail(GBCFD_ERR_TIMEOUT, "a bounded device wait timed out");
  if (flags) return fail(GBCFD_ERR_NONPHYSICAL, "non-positive density or pressure, or a non-finite value");
  return GBCFD_OK;
}

// ---- learned convergence accelerator ------------------------------------------------------------
using bf16 = __nv_bfloat16;
struct gbcfd_accel_s {
  int nx, ny, nz, batch, zper;
  long long cells;            // batch x nx x ny x nz
  learn::Net net;
  bf16 *x, *a1, *a2, *dy, *dz1, *dz2;
  float *z1, *z2, *y;
  double *R, *qsave, *partial, *stats;
  void* dtlsave;              // gbcfd_accel_try_smooth: the block's local time steps before the try
  DevCtrl* ctrlsave;          // and its control block (time step, norms, flags)
  int pgrid;
  int step_count;
};

static const size_t kAccelParts = 1024;  // rows of the per-CTA reduction partials

static size_t accel_carve(int nx, int ny, int nz, int batch, int nsm, size_t* off) {
  const long long cells = (long long)nx * ny * nz * batch, vol = (long long)nx * ny * nz;
  const int wgrid = 2 * nsm;
  size_t o = 0;
  auto take = [&](int i, size_t bytes) { off[i] = o; o += align256(bytes); };
  take(0, sizeof(float) * learn::NPARAM);                              // w
  take(1, sizeof(float) * learn::NPARAM);                              // m
  take(2, sizeof(float) * learn::NPARAM);                              // v
  take(3, sizeof(float) * learn::NPARAM);                              // grad
  take(4, sizeof(bf16) * learn::NTAP * learn::P1 * learn::P0);         // w1
  take(5, sizeof(bf16) * learn::NTAP * learn::P2 * learn::P1);         // w2
  take(6, sizeof(bf16) * learn::NTAP * 16 * learn::P2);               // w3 (16 wide)
  take(7, sizeof(bf16) * learn::NTAP * learn::P2 * 16);                // w3b
  take(8, sizeof(bf16) * learn::NTAP * learn::P1 * learn::P2);         // w2b
  take(9, sizeof(float) * (learn::P1 + learn::P2 + learn::P3));       // biases
  take(10, sizeof(float) * learn::NPARAM * (size_t)wgrid);             // weight-gradient partials
  take(11, sizeof(bf16) * 16 * cells);                                 // x
  take(12, sizeof(bf16) * 32 * cells);                                 // a1
  take(13, sizeof(bf16) * 32 * cells);                                 // a2
  take(14, sizeof(float) * 32 * cells);                                // z1
  take(15, sizeof(float) * 32 * cells);                                // z2
  take(16, sizeof(float) * 8 * cells);                                 // y
  take(17, sizeof(bf16) * 16 * cells);                                 // dy
  take(18, sizeof(bf16) * 32 * cells);                                 // dz2
  take(19, sizeof(bf16) * 32 * cells);                                 // dz1
  take(20, sizeof(double) * 5 * vol);                                  // R (one volume)
  take(21, sizeof(double) * 5 * vol);                                  // saved state
  take(22, sizeof(double) * NPART * kAccelParts);                      // partials
  take(23, sizeof(double) * 8);                                        // stats
  take(24, sizeof(int) * 4);                                           // timeout flag
  take(25, sizeof(double) * (size_t)make_geometry(nx, ny, nz).field);   // saved local time steps (try_smooth;
                                                                       // >= the f32 field's bytes)
  take(26, sizeof(DevCtrl));                                           // saved control block (try_smooth)
  return o;
}

extern "C" int gbcfd_accel_required_bytes(int nx, int ny, int nz, int batch, size_t* bytes) {
  if (nx < 1 || ny < 1 || nz < 1 || batch < 1) return fail(GBCFD_ERR_ARG, "sizes must be >= 1");
  if (!bytes) return fail(GBCFD_ERR_ARG, "bytes is NULL");
  int dev = 0, nsm = 0;
  int rc = device_sms(&dev, &nsm);
  if (rc) return rc;
  size_t off[27];
  *bytes = accel_carve(nx, ny, nz, batch, nsm, off);
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_create(int nx, int ny, int nz, int batch, int zperiodic, void* dev_mem, size_t bytes,
                                  gbcfd_accel* out) {
  if (!out) return fail(GBCFD_ERR_ARG, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  int rc = gbcfd_accel_required_bytes(nx, ny, nz, batch, &need);
  if (rc) return rc;
  if (!dev_mem) return fail(GBCFD_ERR_ARG, "dev_mem is NULL");
  if (((uintptr_t)dev_mem & 255u) != 0) return fail(GBCFD_ERR_MEMORY, "dev_mem must be 256-byte aligned");
  if (bytes < need) return fail(GBCFD_ERR_MEMORY, "dev_mem smaller than gbcfd_accel_required_bytes");
  int dev = 0, nsm = 0;
  rc = device_sms(&dev, &nsm);
  if (rc) return rc;
  size_t off[27];
  accel_carve(nx, ny, nz, batch, nsm, off);
  char* base = static_cast<char*>(dev_mem);
  gbcfd_accel a = new gbcfd_accel_s();
  a->nx = nx; a->ny = ny; a->nz = nz; a->batch = batch; a->zper = zperiodic ? 1 : 0;
  a->cells = (long long)nx * ny * nz * batch;
  learn::Net& n = a->net;
  n.w = reinterpret_cast<float*>(base + off[0]);
  n.m = reinterpret_cast<float*>(base + off[1]);
  n.v = reinterpret_cast<float*>(base + off[2]);
  n.grad = reinterpret_cast<float*>(base + off[3]);
  n.w1 = reinterpret_cast<bf16*>(base + off[4]);
  n.w2 = reinterpret_cast<bf16*>(base + off[5]);
  n.w3 = reinterpret_cast<bf16*>(base + off[6]);
  n.w3b = reinterpret_cast<bf16*>(base + off[7]);
  n.w2b = reinterpret_cast<bf16*>(base + off[8]);
  n.b1 = reinterpret_cast<float*>(base + off[9]);
  n.b2 = n.b1 + learn::P1;
  n.b3 = n.b2 + learn::P2;
  n.wpart = reinterpret_cast<float*>(base + off[10]);
  n.wgrid = 2 * nsm;
  a->x = reinterpret_cast<bf16*>(base + off[11]);
  a->a1 = reinterpret_cast<bf16*>(base + off[12]);
  a->a2 = reinterpret_cast<bf16*>(base + off[13]);
  a->z1 = reinterpret_cast<float*>(base + off[14]);
  a->z2 = reinterpret_cast<float*>(base + off[15]);
  a->y = reinterpret_cast<float*>(base + off[16]);
  a->dy = reinterpret_cast<bf16*>(base + off[17]);
  a->dz2 = reinterpret_cast<bf16*>(base + off[18]);
  a->dz1 = reinterpret_cast<bf16*>(base + off[19]);
  a->R = reinterpret_cast<double*>(base + off[20]);
  a->qsave = reinterpret_cast<double*>(base + off[21]);
  a->partial = reinterpret_cast<double*>(base + off[22]);
  a->stats = reinterpret_cast<double*>(base + off[23]);
  n.flag = reinterpret_cast<int*>(base + off[24]);
  a->dtlsave = base + off[25];
  a->ctrlsave = reinterpret_cast<DevCtrl*>(base + off[26]);
  a->pgrid = (int)std::min<size_t>(kAccelParts, (size_t)4 * nsm);
  a->step_count = 0;
  cudaError_t e = cudaMemset(base, 0, off[11]);  // parameters, moments, packed weights: zero
  if (e == cudaSuccess) e = cudaMemset(n.flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { delete a; return cuda_fail(e, "initialising the accelerator"); }
  *out = a;
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_destroy(gbcfd_accel a) {
  if (!a) return fail(GBCFD_ERR_ARG, "accelerator is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  delete a;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_set_params(gbcfd_accel a, const float* params, void* stream) {
  if (!a || !params) return fail(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(a->net.w, params, sizeof(float) * learn::NPARAM, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(a->net.m, 0, sizeof(float) * learn::NPARAM, s));
  CK(cudaMemsetAsync(a->net.v, 0, sizeof(float) * learn::NPARAM, s));
  CK(cudaMemsetAsync(a->net.grad, 0, sizeof(float) * learn::NPARAM, s));
  CK(learn::launch_pack(a->net, s));
  CK(cudaStreamSynchronize(s));
  a->step_count = 0;
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_get_params(gbcfd_accel a, float* params, void* stream) {
  if (!a || !params) return fail(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(params, a->net.w, sizeof(float) * learn::NPARAM, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_get_train_state(gbcfd_accel a, float* grad, float* m, float* v, void* stream) {
  if (!a) return fail(GBCFD_ERR_ARG, "accelerator is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(float) * learn::NPARAM;
  if (grad) CK(cudaMemcpyAsync(grad, a->net.grad, bytes, cudaMemcpyDeviceToHost, s));
  if (m) CK(cudaMemcpyAsync(m, a->net.m, bytes, cudaMemcpyDeviceToHost, s));
  if (v) CK(cudaMemcpyAsync(v, a->net.v, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GBCFD_OK;
}

static learn::ConvArgs conv_args(gbcfd_accel a, const void* in, const bf16* w, const float* bias, void* out,
                                 float* zsave, const float* zprev) {
  learn::ConvArgs c;
  c.in = static_cast<const bf16*>(in);
  c.w = w;
  c.bias = bias;
  c.out = out;
  c.zsave = zsave;
  c.zprev = zprev;
  c.X = a->nx; c.Y = a->ny; c.Z = a->nz; c.B = a->batch; c.zper = a->zper;
  return c;
}

// the three forward convolutions; z1, z2 kept when training
static int accel_forward(gbcfd_accel a, const void* x, float* y, bool keep, cudaStream_t s) {
  const learn::Net& n = a->net;
  CK(learn::launch_conv(1, learn::FWD_SILU, conv_args(a, x, n.w1, n.b1, a->a1, keep ? a->z1 : nullptr, nullptr),
                        n.flag, s));
  CK(learn::launch_conv(2, learn::FWD_SILU, conv_args(a, a->a1, n.w2, n.b2, a->a2, keep ? a->z2 : nullptr, nullptr),
                        n.flag, s));
  CK(learn::launch_conv(3, learn::FWD_LINEAR, conv_args(a, a->a2, n.w3, n.b3, y, nullptr, nullptr), n.flag, s));
  return GBCFD_OK;
}

static int check_dev(const void* p, const char* what) {
  bool dev = false;
  int rc = is_device_ptr(p, &dev);
  if (rc) return rc;
  if (!dev) return fail(GBCFD_ERR_ARG, std::string(what) + " must be device memory");
  if (((uintptr_t)p & 15u) != 0) return fail(GBCFD_ERR_ARG, std::string(what) + " must be 16-byte aligned");
  return GBCFD_OK;
}

// report (and clear) a timeout flagged by a convolution's bounded wait; synchronises the stream
static int accel_flag(gbcfd_accel a, cudaStream_t s) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, a->net.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h) {
    CK(cudaMemsetAsync(a->net.flag, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return fail(GBCFD_ERR_TIMEOUT, "a tensor-core convolution's bounded wait timed out");
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_forward(gbcfd_accel a, const void* x, float* y, void* stream) {
  if (!a || !x || !y) return fail(GBCFD_ERR_ARG, "NULL argument");
  int rc = check_dev(x, "x");
  if (!rc) rc = check_dev(y, "y");
  if (rc) return rc;
  rc = accel_forward(a, x, y, false, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return accel_flag(a, static_cast<cudaStream_t>(stream));
}

extern "C" int gbcfd_accel_train_step(gbcfd_accel a, const void* x, const float* t, float lr, int step, double* loss,
                                      void* stream) {
  if (!a || !x || !t) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (step < 1) return fail(GBCFD_ERR_ARG, "step counts from 1");
  int rc = check_dev(x, "x");
  if (!rc) rc = check_dev(t, "t");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const learn::Net& n = a->net;
  rc = accel_forward(a, x, a->y, true, s);
  if (rc) return rc;
  CK(learn::launch_loss(a->y, t, a->dy, a->partial, a->cells, a->pgrid, s));
  CK(learn::launch_sum(a->partial, a->pgrid, 1, a->stats + 4, s));
  CK(learn::launch_wgrad(3, a->a2, a->dy, n, a->nx, a->ny, a->nz, a->batch, a->zper, s));
  CK(learn::launch_conv(3, learn::BWD_DSILU, conv_args(a, a->dy, n.w3b, nullptr, a->dz2, nullptr, a->z2), n.flag, s));
  CK(learn::launch_wgrad(2, a->a1, a->dz2, n, a->nx, a->ny, a->nz, a->batch, a->zper, s));
  CK(learn::launch_conv(2, learn::BWD_DSILU, conv_args(a, a->dz2, n.w2b, nullptr, a->dz1, nullptr, a->z1), n.flag, s));
  CK(learn::launch_wgrad(1, static_cast<const bf16*>(x), a->dz1, n, a->nx, a->ny, a->nz, a->batch, a->zper, s));
  CK(learn::launch_grad_reduce(n, s));
  CK(learn::launch_adam(n, lr, step, s));
  CK(learn::launch_pack(n, s));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, a->stats + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (loss) *loss = h / (5.0 * (double)a->cells);
  return accel_flag(a, s);
}

// the block as the feature kernels see it
static int accel_view(gbcfd_accel a, gbcfd_block b, learn::BlockView* v) {
  if (!b) return fail(GBCFD_ERR_ARG, "block is NULL");
  if (b->nx != a->nx || b->ny != a->ny || b->nz != a->nz) return fail(GBCFD_ERR_ARG, "block size differs from the accelerator's volume");
  if (!b->has_state) return fail(GBCFD_ERR_STATE, "block has no state");
  if (b->next_stage != 1) return fail(GBCFD_ERR_STATE, "block is between stages");
  int far = -1;
  for (int f = 0; f < 6; ++f)
    if (b->bc_kind[f] == GBCFD_BC_FARFIELD && !b->nbr[f]) far = f;
  if (far < 0) return fail(GBCFD_ERR_ARG, "the block has no far-field face (the free stream scales the features)");
  const double* inf = b->bc_inf;
  const double gm = b->p.gamma, c = std::sqrt(gm * inf[4] / inf[0]);
  v->nx = b->nx; v->ny = b->ny; v->nz = b->nz;
  v->field = b->g.field; v->fieldf = b->g.fieldf;
  v->px = b->g.px; v->pxf = b->g.pxf;
  v->q = state_ptr(b);
  v->sh = b->p.precision == GBCFD_MIXED ? b->sh[b->cur] : nullptr;
  v->dtl = b->dtl;
  v->dtl_f32 = b->p.precision == GBCFD_MIXED;
  v->dt = &b->ctrl->dt;
  v->qinf[0] = inf[0];
  v->qinf[1] = inf[0] * inf[1];
  v->qinf[2] = inf[0] * inf[2];
  v->qinf[3] = inf[0] * inf[3];
  v->qinf[4] = inf[4] / (gm - 1.0) + 0.5 * inf[0] * (inf[1] * inf[1] + inf[2] * inf[2] + inf[3] * inf[3]);
  v->ref[0] = inf[0];
  v->ref[1] = v->ref[2] = v->ref[3] = inf[0] * c;
  v->ref[4] = inf[0] * c * c;
  return GBCFD_OK;
}

// residual of the block's current state into a->R and its statistics into a->stats[at], [at+1]
static int accel_residual_stats(gbcfd_accel a, gbcfd_block b, const learn::BlockView& v, int at, cudaStream_t s) {
  int rc = prepare_metrics(&b, 1, s);
  if (rc) return rc;
  rc = exchange(&b, 1, F_STATE, true, s);
  if (rc) return rc;
  rc = run_stage(b, 0, a->R, s);
  if (rc) return rc;
  CK(learn::launch_feature_stats(v, a->R, a->partial, a->pgrid, s));
  CK(learn::launch_sum(a->partial, a->pgrid, 2, a->stats + at, s));
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_features(gbcfd_accel a, gbcfd_block b, void* x, void* stream) {
  if (!a) return fail(GBCFD_ERR_ARG, "accelerator is NULL");
  if (x) {
    int rc = check_dev(x, "x");
    if (rc) return rc;
  }
  learn::BlockView v;
  int rc = accel_view(a, b, &v);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = accel_residual_stats(a, b, v, 0, s);
  if (rc) return rc;
  CK(learn::launch_features(v, a->R, a->stats, x ? static_cast<bf16*>(x) : a->x, a->qsave, s));
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_target(gbcfd_accel a, gbcfd_block b, float* t, void* stream) {
  if (!a || !t) return fail(GBCFD_ERR_ARG, "NULL argument");
  int rc = check_dev(t, "t");
  if (rc) return rc;
  learn::BlockView v;
  rc = accel_view(a, b, &v);
  if (rc) return rc;
  CK(learn::launch_target(v, a->qsave, a->stats, t, static_cast<cudaStream_t>(stream)));
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_try(gbcfd_accel a, gbcfd_block b, void* stream, int* accepted, double norms[2]) {
  if (!a || !accepted) return fail(GBCFD_ERR_ARG, "NULL argument");
  learn::BlockView v;
  int rc = accel_view(a, b, &v);
  if (rc) return rc;
  if (a->batch != 1) return fail(GBCFD_ERR_ARG, "an accelerator for one volume is needed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = accel_residual_stats(a, b, v, 0, s);
  if (rc) return rc;
  CK(learn::launch_features(v, a->R, a->stats, a->x, a->qsave, s));
  rc = accel_forward(a, a->x, a->y, false, s);
  if (rc) return rc;
  CK(learn::launch_apply(v, a->y, a->qsave, a->stats, 0, s));
  rc = accel_residual_stats(a, b, v, 2, s);
  if (rc) return rc;
  double h[4];
  CK(cudaMemcpyAsync(h, a->stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  rc = accel_flag(a, s);
  if (rc) {  // restore the state before reporting
    CK(learn::launch_apply(v, a->y, a->qsave, a->stats, 1, s));
    int rc2 = init_rate(b, s);
    return rc2 ? rc2 : rc;
  }
  const double n = (double)b->nx * b->ny * b->nz;
  const double r0 = std::sqrt(h[1] / n), r1 = std::sqrt(h[3] / n);
  const bool keep = std::isfinite(r1) && r1 < r0;
  if (keep) {  // the time steps of the new state
    rc = init_rate(b, s);
    if (rc) return rc;
  } else {     // the state back, bit for bit; nothing else of the block was changed
    CK(learn::launch_apply(v, a->y, a->qsave, a->stats, 1, s));
  }
  CK(cudaStreamSynchronize(s));
  *accepted = keep ? 1 : 0;
  if (norms) { norms[0] = r0; norms[1] = r1; }
  return GBCFD_OK;
}

extern "C" int gbcfd_accel_try_smooth(gbcfd_accel a, gbcfd_block b, double alpha, int nsteps, double ratio,
                                      void* stream, int* accepted, double norms[2]) {
  if (!a || !accepted) return fail(GBCFD_ERR_ARG, "NULL argument");
  if (!(alpha > 0.0) || !(alpha <= 4.0)) return fail(GBCFD_ERR_ARG, "alpha must be in (0, 4]");
  if (nsteps < 0 || nsteps > 1000) return fail(GBCFD_ERR_ARG, "nsteps must be 0..1000");
  if (!(ratio > 0.0)) return fail(GBCFD_ERR_ARG, "ratio must be positive");
  if (ratio > 1.0) ratio = 1.0;  // kept only if the residual drops
  learn::BlockView v;
  int rc = accel_view(a, b, &v);
  if (rc) return rc;
  if (a->batch != 1) return fail(GBCFD_ERR_ARG, "an accelerator for one volume is needed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the local time steps: one padded field in the path's flux type (f32 rows have their own pitch)
  const size_t dtl_bytes = b->p.precision == GBCFD_MIXED ? sizeof(float) * (size_t)b->g.fieldf
                                                         : sizeof(double) * (size_t)b->g.field;
  // what the plain steps change besides the state: the control block and the local time steps
  CK(cudaMemcpyAsync(a->ctrlsave, b->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToDevice, s));
  if (b->dtl) CK(cudaMemcpyAsync(a->dtlsave, b->dtl, dtl_bytes, cudaMemcpyDeviceToDevice, s));
  rc = accel_residual_stats(a, b, v, 0, s);
  if (rc) return rc;
  CK(learn::launch_features(v, a->R, a->stats, a->x, a->qsave, s));
  rc = accel_forward(a, a->x, a->y, false, s);
  if (rc) return rc;
  CK(learn::launch_apply(v, a->y, a->qsave, a->stats, 0, s, alpha));
  rc = init_rate(b, s);  // time steps of the predicted state
  if (!rc && nsteps > 0) rc = gbcfd_step(&b, 1, nsteps, stream);
  learn::BlockView w;  // the state's buffers after the steps (the mixed path alternates them)
  if (!rc) rc = accel_view(a, b, &w);
  if (!rc) rc = accel_residual_stats(a, b, w, 2, s);
  int frc = accel_flag(a, s);
  DevCtrl h;
  if (!rc) {
    CK(cudaMemcpyAsync(&h, b->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  }
  double st[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(st, a->stats, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double n = (double)b->nx * b->ny * b->nz;
  const double r0 = std::sqrt(st[1] / n), r1 = std::sqrt(st[3] / n);
  const bool keep = !rc && !frc && h.flag == 0 && std::isfinite(r1) && r1 < ratio * r0;
  if (!keep) {  // the state, time steps and control block back, bit for bit
    if (rc) {   // a failure inside: the views may be stale, take the block's own
      learn::BlockView u;
      if (accel_view(a, b, &u) == GBCFD_OK) w = u; else w = v;
    }
    CK(learn::launch_apply(w, a->y, a->qsave, a->stats, 1, s));
    if (b->dtl) CK(cudaMemcpyAsync(b->dtl, a->dtlsave, dtl_bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(b->ctrl, a->ctrlsave, sizeof(DevCtrl), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  if (rc) return rc;
  if (frc) return frc;
  *accepted = keep ? 1 : 0;
  if (norms) { norms[0] = r0; norms[1] = r1; }
  return GBCFD_OK;
}

// ---- dispatch ----------------------------------------------------------------------------
namespace gbcfd {
cudaError_t launch_stage(int precision, int viscous, int curvi, int stage, const GroupParams& P, int grid,
                         cudaStream_t s, int ty) {
  if (P.push && (stage == 1 || stage == 2)) {  // the folded halo exchange: Cartesian Euler groups
    if (viscous || curvi) return cudaErrorInvalidValue;
    return precision == GBCFD_MIXED ? launch_stage_f32_push(stage, ty, P, grid, s)
                                    : launch_stage_f64_push(stage, ty, P, grid, s);
  }
  if (ty != TY_DEFAULT) {  // the second height: Cartesian Euler blocks only
    if (viscous || curvi) return cudaErrorInvalidValue;
    if (precision == GBCFD_MIXED && ty == TY_ALT_F32) return launch_stage_f32_alt(stage, P, grid, s);
    if (precision == GBCFD_FP64 && ty == TY_ALT_F64) return launch_stage_f64_alt(stage, P, grid, s);
    return cudaErrorInvalidValue;
  }
  if (precision == GBCFD_MIXED)
    return curvi ? launch_stage_f32c(viscous, stage, P, grid, s) : launch_stage_f32(viscous, stage, P, grid, s);
  return curvi ? launch_stage_f64c(viscous, stage, P, grid, s) : launch_stage_f64(viscous, stage, P, grid, s);
}

int stage_tiles(int precision, int viscous, int curvi, int* ty) {
  ty[0] = TY_DEFAULT;
  if (viscous || curvi) return 1;
  ty[1] = precision == GBCFD_MIXED ? TY_ALT_F32 : TY_ALT_F64;
  return 2;
}

int stage_occupancy_tile(int precision, int viscous, int curvi, int ty) {
  if (ty != TY_DEFAULT) return precision == GBCFD_MIXED ? stage_occupancy_f32_alt() : stage_occupancy_f64_alt();
  return precision == GBCFD_MIXED ? (curvi ? stage_occupancy_f32c(viscous) : stage_occupancy_f32(viscous))
                                  : (curvi ? stage_occupancy_f64c(viscous) : stage_occupancy_f64(viscous));
}

cudaError_t stage_prepare_tile(int precision, int viscous, int curvi, int ty) {
  if (ty != TY_DEFAULT) return precision == GBCFD_MIXED ? stage_prepare_f32_alt() : stage_prepare_f64_alt();
  return precision == GBCFD_MIXED ? (curvi ? stage_prepare_f32c(viscous) : stage_prepare_f32(viscous))
                                  : (curvi ? stage_prepare_f64c(viscous) : stage_prepare_f64(viscous));
}
}  // namespace gbcfd

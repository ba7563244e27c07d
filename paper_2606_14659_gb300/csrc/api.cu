// api.cu — the C ABI of librsb (include/rsb.h) and the level driver of
// Recursive Spectral Bisection (paper §4, Algorithm 1).
//
// One call runs every mesh of a batch level by level.  At each level all
// segments (subgraphs) that still own two or more parts are bisected
// together:
//   1. components of every segment (union-find); a segment that fell apart
//      places whole components left in order of their smallest gid and only
//      the straddling component is solved (reading R8);
//   2. one Fiedler problem ("unit") per segment is solved for all units at
//      once — Lanczos (§6) or inverse iteration with CG (§7), FP64 or FP32
//      with an FP64 polish — and, under RESOLVE, deflated solves detect a
//      repeated lambda_2 whose basis is rotated to the quartic minimiser
//      (reading R5, §9);
//   3. every candidate vector is oriented (R4) and split at the proportional
//      count (R6) with the tie window (R7); the candidate with the least
//      weighted cut wins;
//   4. both halves are compacted into the next level's graph (R2).
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rsb_internal.cuh"

// defined in select.cu / solver.cu / graph.cu (not all in the shared header)
int launch_orient(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                  const uint64_t* ckey, const double* v, int cand, double tie_rel,
                  double* partials, cudaStream_t s, int fixed_sign = 0);
int launch_select(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                  const uint64_t* ckey, const double* v, int mode, int cand, int* hist,
                  cudaStream_t s);
int launch_split_below(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                       const uint64_t* ckey, const double* v, int cand, double* partials,
                       cudaStream_t s);
int launch_choose(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                  const uint64_t* ckey, const uint8_t* side, int cb, double* partials,
                  cudaStream_t s);
int launch_finalize_side(const LevelGraph& G, const uint8_t* seg_split,
                         const uint64_t* seg_keystar, const int32_t* seg_unit, const Unit* units,
                         const uint64_t* ckey, uint8_t* side, cudaStream_t s);
int launch_cut(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
               const uint64_t* ckey, const uint8_t* side, int cand, double* partials,
               cudaStream_t s);
int launch_cc_spread(const LevelGraph& G, const int32_t* parent, const uint64_t* cmin,
                     uint64_t* ckey, int* flag, cudaStream_t s);
int solver_setup(Unit* units, int nunits, int nd, int krylov, int maxcycles, double tol,
                 int require_cluster, int keep, SolveBufs& B, cudaStream_t s,
                 long long dim_lo = 0, long long dim_hi = (1ll << 62));
int solver_block_lanczos(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                         int nunits, const uint64_t* ckey, SolveBufs& SB, int f32, int M, int bw,
                         int keep, uint64_t seedbase, int use_graph, cudaStream_t s);
size_t blk_unit_bytes();
int solver_lanczos(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                   const uint64_t* ckey, SolveBufs& B, int f32, int M, uint64_t sd,
                   const double* from64, const float* from32, int use_graph, cudaStream_t s);
int solver_inverse(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                   const uint64_t* ckey, SolveBufs& B, int f32, uint64_t sd, const double* from64,
                   const float* from32, double cg_tol, int cg_maxit, int max_outer, int use_graph,
                   cudaStream_t s, const std::vector<Unit>* amg_units);
void amg_release();
int solver_write_vector(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                        const uint64_t* ckey, SolveBufs& B, int f32, int from_x, double* out,
                        int cand, int better_only, cudaStream_t s);
int solver_keep_better(Unit* units, int nunits, int cand, double tol1, cudaStream_t s);
int solver_quartic(const Tile* tiles, int ntiles, Unit* units, int nunits, const uint64_t* ckey,
                   double* v0, double* v1, double* v2, double* partials, double* mom,
                   cudaStream_t s);
int solver_cluster_check(Unit* units, int nunits, int nd, double cluster_tol, cudaStream_t s);
int solver_stats(const Unit* units, int nunits, int* capped, double* resid_max, cudaStream_t s);
int solver_sum_inner(const Unit* units, int nunits, long long* inner, cudaStream_t s);
int solver_rq_refine(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                     const uint64_t* ckey, SolveBufs& B, const float* from32, cudaStream_t s);

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
static std::string g_detail;
static long long g_launches = 0;

int rsb_set_cuda_error(cudaError_t e, const char* where) {
  g_detail = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? RSB_ENOMEM : RSB_ECUDA;
}
int rsb_set_error(int code, const std::string& what) {
  g_detail = what;
  return code;
}
void rsb_count_launch(int k) { g_launches += k; }

// ----------------------------------------------------------------------------
// tracing: with RSB_TRACE=1 in the environment, every level and every solve
// stage prints its wall time (the stream is synchronised at each mark, so a
// traced run is slower; off by default)
// ----------------------------------------------------------------------------
static int trace_on() {
  const char* e = getenv("RSB_TRACE");
  return (e && *e && *e != '0') ? 1 : 0;
}
static std::chrono::steady_clock::time_point g_trace_t0;
static void trace_mark(cudaStream_t s, const char* fmt, ...) {
  if (!trace_on()) return;
  cudaStreamSynchronize(s);
  const auto now = std::chrono::steady_clock::now();
  const double ms = std::chrono::duration<double, std::milli>(now - g_trace_t0).count();
  g_trace_t0 = now;
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  fprintf(stderr, "[rsb] %9.3f ms  %s\n", ms, buf);
}

// ----------------------------------------------------------------------------
// kernel timing (rsb_profile_begin / rsb_profile_end)
// ----------------------------------------------------------------------------
static struct {
  unsigned mask = 0;  // enabled families (bit f for family f)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  std::vector<int> pool_family;
  std::vector<int> free_list, pending;
  bool capturing = false;
  std::vector<int> captured;
  double ms[PROF_NFAM] = {0};
  long long launches[PROF_NFAM] = {0};
  double bytes[PROF_NFAM] = {0};
  unsigned long long* dbytes = nullptr;  // one device counter per family
} g_prof;

static bool prof_on(int family) {
  return family > PROF_NONE && family < PROF_NFAM && (g_prof.mask >> family & 1u);
}

int prof_before(int family, cudaStream_t s) {
  if (!prof_on(family)) return -1;
  int idx;
  if (!g_prof.free_list.empty()) {
    idx = g_prof.free_list.back();
    g_prof.free_list.pop_back();
  } else {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1;
    g_prof.pool.emplace_back(a, b);
    g_prof.pool_family.push_back(0);
    idx = (int)g_prof.pool.size() - 1;
  }
  g_prof.pool_family[idx] = family;
  cudaEventRecordWithFlags(g_prof.pool[idx].first, s,
                           g_prof.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  return idx;
}
void prof_after(int idx, cudaStream_t s) {
  if (idx < 0) return;
  cudaEventRecordWithFlags(g_prof.pool[idx].second, s,
                           g_prof.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  if (g_prof.capturing) g_prof.captured.push_back(idx);
  else g_prof.pending.push_back(idx);
}
void prof_collect() {
  for (int idx : g_prof.pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_prof.pool[idx].first, g_prof.pool[idx].second) == cudaSuccess) {
      const int f = g_prof.pool_family[idx];
      g_prof.ms[f] += t;
      g_prof.launches[f] += 1;
    } else {
      cudaGetLastError();
    }
  }
  g_prof.pending.clear();
}
void prof_capture_begin() {
  g_prof.capturing = true;
  g_prof.captured.clear();
}
std::vector<int> prof_capture_end() {
  g_prof.capturing = false;
  std::vector<int> v;
  v.swap(g_prof.captured);
  return v;
}
void prof_replay(const std::vector<int>& pairs) {
  g_prof.pending.insert(g_prof.pending.end(), pairs.begin(), pairs.end());
}

unsigned long long* prof_bytes(int family) {
  if (!prof_on(family) || !g_prof.dbytes) return nullptr;
  return g_prof.dbytes + family;
}

extern "C" void rsb_profile_begin(int family) {
  if (family == RSB_PROF_ALL) g_prof.mask = ((1u << PROF_NFAM) - 1u) & ~1u;
  else g_prof.mask = (family > PROF_NONE && family < PROF_NFAM) ? (1u << family) : 0u;
  for (int f = 0; f < PROF_NFAM; ++f) {
    g_prof.ms[f] = 0.0;
    g_prof.launches[f] = 0;
    g_prof.bytes[f] = 0.0;
  }
  g_prof.pending.clear();
  // pairs held by graphs that were destroyed are free again
  g_prof.free_list.clear();
  for (int i = 0; i < (int)g_prof.pool.size(); ++i) g_prof.free_list.push_back(i);
  const size_t nb = sizeof(unsigned long long) * PROF_NFAM;
  if (!g_prof.dbytes && cudaMalloc(&g_prof.dbytes, nb) != cudaSuccess) {
    cudaGetLastError();
    g_prof.dbytes = nullptr;
  }
  if (g_prof.dbytes) cudaMemset(g_prof.dbytes, 0, nb);
}

extern "C" void rsb_profile_end(double* ms_total, int64_t* launches, double* bytes_total) {
  cudaDeviceSynchronize();
  prof_collect();
  unsigned long long b[PROF_NFAM] = {0};
  if (g_prof.dbytes) cudaMemcpy(b, g_prof.dbytes, sizeof(b), cudaMemcpyDeviceToHost);
  double ms = 0.0, by = 0.0;
  long long nl = 0;
  for (int f = 0; f < PROF_NFAM; ++f) {
    g_prof.bytes[f] = (double)b[f];
    ms += g_prof.ms[f];
    nl += g_prof.launches[f];
    by += g_prof.bytes[f];
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = nl;
  if (bytes_total) *bytes_total = by;
  g_prof.mask = 0;
}

extern "C" void rsb_profile_read(int family, double* ms, int64_t* launches, double* bytes) {
  const bool ok = family > PROF_NONE && family < PROF_NFAM;
  if (ms) *ms = ok ? g_prof.ms[family] : 0.0;
  if (launches) *launches = ok ? g_prof.launches[family] : 0;
  if (bytes) *bytes = ok ? g_prof.bytes[family] : 0.0;
}

int devbuf_reserve(DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return RSB_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 8 + 256;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return rsb_set_error(RSB_ENOMEM, std::string("cudaMalloc of ") + std::to_string(want) +
                                         " bytes failed: " + cudaGetErrorString(e));
  }
  b.cap = want;
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// workspace
// ----------------------------------------------------------------------------
struct PrecBufs {
  DevBuf Q, W0, W1, Y, X, R, P, AP;
  DevBuf Z0, Z1;  // block Lanczos: interleaved residual blocks
};

struct Ctx {
  int device = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // level graphs (double-buffered)
  DevBuf slice_ptr[2], ent[2], deg[2], gid[2], home[2], row_seg[2];
  DevBuf len, slice_sz, scan_tmp, tmp64, newpos;
  DevBuf parent, cmin, ckey, side;
  DevBuf units, tiles, sunits, stiles;
  DevBuf hist, partials, mom, sbuf, blk;
  DevBuf cand[3];
  PrecBufs pb[2];  // 0: FP64, 1: FP32
  DevBuf seg_row0, seg_nleft, seg_child0, seg_p0, seg_split, seg_keystar, seg_unit, seg_ncomp;
  DevBuf counters;  // one Counters record
  DevBuf coords_cat;            // RCB: (x, y, z) per element, caller order, meshes concatenated
  DevBuf perm, iperm, rcb_home;  // RCB reordering: new row -> caller row and back
  // gather-scatter (element -> vertex ids): buckets of elements per vertex
  DevBuf gs_count, gs_cursor, gs_bptr, gs_bucket, gs_ev32, gs_len, gs_rowptr, gs_w, gs_misc;
  DevBuf part_concat;
  int trmax = 0;    // largest tile of the level being solved, rows
  std::vector<DevBuf> stage;  // staged host inputs
  int* h_pinned = nullptr;
};

static Ctx* g_ctx[64] = {nullptr};

static void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

static int ctx_get(Ctx** out) {
  int dev = 0;
  RSB_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return rsb_set_error(RSB_EINVAL, "device index");
  if (!g_ctx[dev]) {
    Ctx* c = new Ctx();
    c->device = dev;
    RSB_CK(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
    RSB_CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    RSB_CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    RSB_CK(cudaMallocHost(&c->h_pinned, 64));
    g_ctx[dev] = c;
  }
  *out = g_ctx[dev];
  return RSB_OK;
}

struct Counters {
  int flag;
  int n_active;
  int n_cg;
  int capped;
  long long cycles;
  double resid_max;
  GridBar gb;
  int jmin[2];
  long long inner;  // CG iterations of the inverse-iteration solves
};

// ----------------------------------------------------------------------------
// pointer staging (host inputs are copied in, host outputs copied back)
// ----------------------------------------------------------------------------
static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static int stage_in(Ctx& c, const T* p, size_t count, const T** out) {
  if (!p || count == 0 || is_device_ptr(p)) {
    *out = p;
    return RSB_OK;
  }
  c.stage.emplace_back();
  DevBuf& b = c.stage.back();
  int rc = devbuf_reserve(b, sizeof(T) * count);
  if (rc) return rc;
  RSB_CK(cudaMemcpyAsync(b.p, p, sizeof(T) * count, cudaMemcpyHostToDevice, c.s));
  *out = (const T*)b.p;
  return RSB_OK;
}

static void stage_clear(Ctx& c) {
  for (auto& b : c.stage) free_buf(b);
  c.stage.clear();
}

// ----------------------------------------------------------------------------
// options
// ----------------------------------------------------------------------------
extern "C" void rsb_options_default(rsb_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->method = RSB_LANCZOS;
  o->precision = RSB_FP64;
  o->krylov_dim = 40;
  o->max_restarts = 50;
  o->tol = 1e-10;
  o->cg_tol = 1e-12;
  o->cg_maxit = 4000;
  o->max_outer = 50;
  o->seed = 0x5EED;
  o->degenerate_policy = RSB_DEGEN_RESOLVE;
  o->cluster_tol = 0.05;
  o->tie_rel = 1e-5;
  o->mixed_tol = 1e-6;
  o->batched = 1;
  o->use_graph = 3;
  o->validate = 0;
  o->polish_cycles = 2;
  o->keep = 8;
  o->tile_rows = 0;
  o->polish_dim = 16;
  o->block = 1;
  o->reorder = 0;
  o->amg = 0;
}

static int check_options(const rsb_options& o) {
  if (o.method != RSB_LANCZOS && o.method != RSB_INVERSE && o.method != RSB_RCB)
    return rsb_set_error(RSB_EINVAL, "method");
  if (o.reorder != 0 && o.reorder != 1) return rsb_set_error(RSB_EINVAL, "reorder");
  if (o.amg != 0 && o.amg != 1) return rsb_set_error(RSB_EINVAL, "amg");
  if (o.precision != RSB_FP64 && o.precision != RSB_MIXED)
    return rsb_set_error(RSB_EINVAL, "precision");
  if (o.krylov_dim < 1 || o.krylov_dim > RSB_MAXM) return rsb_set_error(RSB_EINVAL, "krylov_dim");
  if (o.keep < 0 || o.keep > RSB_MAXKEEP) return rsb_set_error(RSB_EINVAL, "keep");
  if (o.tile_rows < 0 || o.tile_rows > 64) return rsb_set_error(RSB_EINVAL, "tile_rows");
  if (o.polish_dim < 2 || o.polish_dim > RSB_MAXM) return rsb_set_error(RSB_EINVAL, "polish_dim");
  if (o.block < 1 || o.block > 4) return rsb_set_error(RSB_EINVAL, "block");
  if (o.use_graph < 0 || o.use_graph > 3) return rsb_set_error(RSB_EINVAL, "use_graph");
  if (o.max_restarts < 1) return rsb_set_error(RSB_EINVAL, "max_restarts");
  if (!(o.tol > 0) || !(o.cg_tol > 0) || !(o.mixed_tol > 0))
    return rsb_set_error(RSB_EINVAL, "tolerances");
  if (o.cg_maxit < 1 || o.max_outer < 1 || o.polish_cycles < 0)
    return rsb_set_error(RSB_EINVAL, "iteration caps");
  if (!(o.cluster_tol >= 0) || !(o.tie_rel >= 0)) return rsb_set_error(RSB_EINVAL, "cluster/tie");
  if (o.degenerate_policy != RSB_DEGEN_NONE && o.degenerate_policy != RSB_DEGEN_RESOLVE)
    return rsb_set_error(RSB_EINVAL, "degenerate_policy");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// level-0 ingest of one or several meshes
// ----------------------------------------------------------------------------
struct MeshIn {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* wt;
  const int64_t* gid;
  const double* coords;
  int64_t nnz;
};

// perm / iperm (optional, meshes concatenated, indices local to each mesh): row
// i of mesh m in the level-0 graph is the caller's row perm[off_m + i], and the
// caller's row j becomes row iperm[off_m + j]
static int build_level0(Ctx& c, const std::vector<MeshIn>& meshes, int validate, LevelGraph& G,
                        const int64_t* perm = nullptr, const int32_t* iperm = nullptr) {
  int64_t N = 0;
  for (auto& m : meshes) N += m.n;
  if (N >= RSB_MAXN) return rsb_set_error(RSB_EINVAL, "too many rows (limit 2^29)");
  const int64_t nsl = (N + 31) / 32;
  int rc;
  if ((rc = devbuf_reserve(c.len, sizeof(int32_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.slice_sz, sizeof(int64_t) * (nsl + 2)))) return rc;
  if ((rc = devbuf_reserve(c.scan_tmp, scan_tmp_bytes(std::max<int64_t>(N, nsl) + 2)))) return rc;
  if ((rc = devbuf_reserve(c.slice_ptr[0], sizeof(int64_t) * (nsl + 2)))) return rc;
  if ((rc = devbuf_reserve(c.counters, 256))) return rc;
  RSB_CK(cudaMemsetAsync(c.counters.p, 0, 256, c.s));
  int* flag = &dptr<Counters>(c.counters)->flag;
  int64_t off = 0;
  for (auto& m : meshes) {
    if ((rc = launch_validate(m.row_ptr, m.col, m.wt, m.n, validate, flag, c.s))) return rc;
    if ((rc = launch_row_lengths(m.row_ptr, m.n, dptr<int32_t>(c.len) + off, c.s,
                                 perm ? perm + off : nullptr)))
      return rc;
    off += m.n;
  }
  RSB_CK(cudaMemcpyAsync(c.h_pinned, flag, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  if (c.h_pinned[0]) {
    const int f = c.h_pinned[0];
    std::string why = "invalid graph:";
    if (f & 1) why += " row_ptr";
    if (f & 2) why += " column out of range";
    if (f & 4) why += " self loop";
    if (f & 8) why += " weight outside 1..7";
    if (f & 16) why += " asymmetric";
    return rsb_set_error(RSB_EINVAL, why);
  }
  if ((rc = launch_slice_widths(dptr<int32_t>(c.len), N, dptr<int64_t>(c.slice_sz), c.s))) return rc;
  RSB_CK(cudaMemsetAsync(dptr<int64_t>(c.slice_sz) + nsl, 0, sizeof(int64_t), c.s));
  if ((rc = launch_scan_i64(dptr<int64_t>(c.slice_sz), dptr<int64_t>(c.slice_ptr[0]), nsl + 1,
                            c.scan_tmp.p, c.scan_tmp.cap, c.s)))
    return rc;
  int64_t total = 0;
  RSB_CK(cudaMemcpyAsync(&total, dptr<int64_t>(c.slice_ptr[0]) + nsl, sizeof(int64_t),
                         cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  if ((rc = devbuf_reserve(c.ent[0], sizeof(uint32_t) * (size_t)std::max<int64_t>(total, 1)))) return rc;
  for (int k = 0; k < 2; ++k) {
    if ((rc = devbuf_reserve(c.deg[k], sizeof(int32_t) * (N + 32)))) return rc;
    if ((rc = devbuf_reserve(c.gid[k], sizeof(int64_t) * (N + 32)))) return rc;
    if ((rc = devbuf_reserve(c.home[k], sizeof(int64_t) * (N + 32)))) return rc;
    if ((rc = devbuf_reserve(c.row_seg[k], sizeof(int32_t) * (N + 32)))) return rc;
  }
  if ((rc = devbuf_reserve(c.slice_ptr[1], sizeof(int64_t) * (nsl + 2)))) return rc;
  G.n = (int32_t)N;
  G.nslices = nsl;
  G.slice_ptr = dptr<int64_t>(c.slice_ptr[0]);
  G.ent = dptr<uint32_t>(c.ent[0]);
  G.deg = dptr<int32_t>(c.deg[0]);
  G.gid = dptr<int64_t>(c.gid[0]);
  G.home = dptr<int64_t>(c.home[0]);
  G.row_seg = dptr<int32_t>(c.row_seg[0]);
  G.nent = total;
  off = 0;
  for (size_t i = 0; i < meshes.size(); ++i) {
    const MeshIn& m = meshes[i];
    if ((rc = launch_fill_sell(m.row_ptr, m.col, m.wt, m.gid, m.n, off, off, (int32_t)i,
                               G.slice_ptr, G.ent, G.deg, G.gid, G.home, G.row_seg, c.s,
                               perm ? perm + off : nullptr, iperm ? iperm + off : nullptr)))
      return rc;
    off += m.n;
  }
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// tiles
// ----------------------------------------------------------------------------
static int max_tile_rows(const std::vector<Tile>& tiles) {
  int m = 0;
  for (const Tile& t : tiles) m = std::max(m, t.row1 - t.row0);
  return m;
}

// mesh_rows[i]: the element count of the mesh unit i belongs to (empty: the
// units are parts of one mesh, whose rows they cover)
static void make_tiles(std::vector<Unit>& units, std::vector<Tile>& tiles, int rmin = RSB_MINR,
                       const std::vector<int64_t>& mesh_rows = {}) {
  tiles.clear();
  // rows per thread of a tile: at least rmin (memory-level parallelism), more
  // in a mesh so large that one of its levels would exceed about
  // RSB_TARGET_TILES tiles, and more for large units so that a unit has at
  // most RSB_MAXTILES_PER_UNIT tiles.  The rule looks at the unit's own mesh,
  // so a mesh is tiled alike alone and in a batch (same sums, same bits).
  int64_t nall = 0;
  for (const Unit& u : units) nall += u.nrows;
  for (size_t i = 0; i < units.size(); ++i) {
    Unit& u = units[i];
    const int64_t nr = u.nrows;
    const int64_t nmesh = mesh_rows.empty() ? nall : mesh_rows[i];
    const int64_t rmesh = (nmesh + (int64_t)RSB_BLOCK * RSB_TARGET_TILES - 1) /
                          ((int64_t)RSB_BLOCK * RSB_TARGET_TILES);
    int64_t R = (nr + (int64_t)RSB_BLOCK * RSB_MAXTILES_PER_UNIT - 1) /
                ((int64_t)RSB_BLOCK * RSB_MAXTILES_PER_UNIT);
    if (R < rmin) R = rmin;
    if (R < rmesh) R = rmesh;
    const int64_t tr = R * RSB_BLOCK;
    u.tile0 = (int32_t)tiles.size();
    int nt = 0;
    for (int64_t b = 0; b < nr; b += tr) {
      Tile t;
      t.unit = (int32_t)i;
      t.row0 = (int32_t)(u.row0 + b);
      t.row1 = (int32_t)(u.row0 + std::min<int64_t>(nr, b + tr));
      t.pad = 0;
      tiles.push_back(t);
      ++nt;
    }
    u.ntile = nt;
  }
}

static Unit blank_unit() {
  Unit u;
  memset(&u, 0, sizeof(u));
  u.status = U_IDLE;
  u.ncand = 1;
  return u;
}

// ----------------------------------------------------------------------------
// solver buffers
// ----------------------------------------------------------------------------
static int reserve_prec(Ctx& c, int f32, int64_t N, int M, SolveBufs& B) {
  PrecBufs& p = c.pb[f32 ? 1 : 0];
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const size_t vb = es * (size_t)(N + 32);
  // basis stride: a multiple of 32 rows with 4 rows to spare, so every vector
  // starts 128-byte aligned and a chunk copy rounded out to 16 bytes stays
  // inside its vector (bulk copies need 16-byte addresses and sizes)
  const int64_t ldN = (N + 4 + 31) / 32 * 32;
  int rc;
  if ((rc = devbuf_reserve(p.Q, es * (size_t)ldN * (size_t)M + 256))) return rc;
  if ((rc = devbuf_reserve(p.W0, vb))) return rc;
  if ((rc = devbuf_reserve(p.W1, vb))) return rc;
  if ((rc = devbuf_reserve(p.Y, vb))) return rc;
  if ((rc = devbuf_reserve(p.X, vb))) return rc;
  if ((rc = devbuf_reserve(p.R, vb))) return rc;
  if ((rc = devbuf_reserve(p.P, vb))) return rc;
  if ((rc = devbuf_reserve(p.AP, vb))) return rc;
  B.Q = p.Q.p;
  B.W0 = p.W0.p;
  B.W1 = p.W1.p;
  B.Y = p.Y.p;
  B.X = p.X.p;
  B.R = p.R.p;
  B.P = p.P.p;
  B.AP = p.AP.p;
  B.N = ldN;
  Counters* cn = dptr<Counters>(c.counters);
  B.n_active = &cn->n_active;
  B.n_cg = &cn->n_cg;
  B.stat_cycles = &cn->cycles;
  B.h_active = c.h_pinned + 4;
  B.gb = &cn->gb;
  B.jmin = cn->jmin;
  B.S = dptr<double>(c.sbuf);
  B.partials = dptr<double>(c.partials);
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// Fiedler solve of every unit of a level for candidate `cand` (nd = cand
// deflation vectors), with the FP64 polish in mixed precision.  Result vector
// in c.cand[cand].
// ----------------------------------------------------------------------------
struct RunStats {
  int64_t solves = 0, cycles = 0, inner = 0;
  int nonconv = 0;
  double resid_max = 0;
};

static int solve_candidate(Ctx& c, const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                           int nunits, int64_t maxn, const rsb_options& o, int cand,
                           RunStats& rs, const std::vector<Unit>& hunits) {
  const int nd = cand;
  const int64_t dim = maxn - 1 - nd;
  if (dim <= 0) return RSB_OK;
  const int M = (int)std::min<int64_t>(o.krylov_dim, dim);
  const uint64_t sd = splitmix64(o.seed + (uint64_t)nd);
  const int mixed = o.precision == RSB_MIXED;
  const int use_graph = o.use_graph;
  const uint64_t* ckey = dptr<uint64_t>(c.ckey);
  int rc;
  SolveBufs B;
  B.trmax = c.trmax;
  B.D[0] = nd > 0 ? dptr<double>(c.cand[0]) : nullptr;
  B.D[1] = nd > 1 ? dptr<double>(c.cand[1]) : nullptr;
  Counters* cn = dptr<Counters>(c.counters);
  double* out = dptr<double>(c.cand[cand]);
  const int require_cluster = nd > 0;
  const int inverse = o.method == RSB_INVERSE;
  // stage 1: working precision
  if ((rc = reserve_prec(c, mixed, G.n, std::max(M, 1), B))) return rc;
  const double tol1 = mixed ? std::max(o.tol, o.mixed_tol) : o.tol;
  RSB_CK(cudaMemsetAsync(&cn->cycles, 0, sizeof(long long), c.s));
  // block Lanczos for the units with room for a full basis and one more block;
  // the single-vector method below takes the rest
  long long single_hi = 1ll << 62;
  if (!inverse && o.block > 1) {
    const long long lo = (long long)o.krylov_dim + o.block;
    single_hi = lo - 1;
    if (dim >= lo) {
      PrecBufs& pb = c.pb[mixed ? 1 : 0];
      const size_t es = mixed ? sizeof(float) : sizeof(double);
      if ((rc = devbuf_reserve(pb.Z0, es * 4 * (size_t)(G.n + 32))) ||
          (rc = devbuf_reserve(pb.Z1, es * 4 * (size_t)(G.n + 32))) ||
          (rc = devbuf_reserve(c.blk, blk_unit_bytes() * (size_t)nunits)))
        return rc;
      B.Z0 = pb.Z0.p;
      B.Z1 = pb.Z1.p;
      B.bu = c.blk.p;
      if ((rc = solver_setup(units, nunits, nd, o.krylov_dim, o.max_restarts, tol1,
                             require_cluster, o.keep, B, c.s, lo, 1ll << 62)))
        return rc;
      if ((rc = solver_block_lanczos(G, tiles, ntiles, units, nunits, ckey, B, mixed,
                                     o.krylov_dim, o.block, o.keep, o.seed + (uint64_t)nd,
                                     use_graph, c.s)))
        return rc;
      trace_mark(c.s, "cand %d stage 1 (block lanczos %d, %s): %d units, %d tiles", cand,
                 o.block, mixed ? "fp32" : "fp64", nunits, ntiles);
    }
  }
  if ((rc = solver_setup(units, nunits, nd, o.krylov_dim, o.max_restarts, tol1, require_cluster,
                         o.keep, B, c.s, 0, single_hi)))
    return rc;
  if (inverse) {
    const double cgt = mixed ? std::max(o.cg_tol, 1e-6) : o.cg_tol;
    rc = solver_inverse(G, tiles, ntiles, units, nunits, ckey, B, mixed, sd, nullptr, nullptr, cgt,
                        o.cg_maxit, o.max_outer, use_graph, c.s, o.amg ? &hunits : nullptr);
    if (!rc) {
      RSB_CK(cudaMemsetAsync(&cn->inner, 0, sizeof(long long), c.s));
      rc = solver_sum_inner(units, nunits, &cn->inner, c.s);
    }
  } else {
    rc = solver_lanczos(G, tiles, ntiles, units, nunits, ckey, B, mixed, M, sd, nullptr, nullptr,
                        use_graph, c.s);
  }
  if (rc) return rc;
  trace_mark(c.s, "cand %d stage 1 (%s %s): %d units, %d tiles", cand,
             inverse ? "inverse" : "lanczos", mixed ? "fp32" : "fp64", nunits, ntiles);
  const void* stage1_vec = inverse ? B.X : B.Y;
  if (!mixed) {
    if ((rc = solver_write_vector(G, tiles, ntiles, units, ckey, B, 0, inverse, out, cand, 0,
                                  c.s)))
      return rc;
  } else {
    // stage 2: FP64 Rayleigh-quotient refinement of the FP32 vector
    SolveBufs B64 = B;
    const int Mp = (int)std::min<int64_t>(o.polish_dim, dim);
    if ((rc = reserve_prec(c, 0, G.n, o.polish_cycles > 0 ? std::max(Mp, 1) : 1, B64))) return rc;
    B64.D[0] = B.D[0];
    B64.D[1] = B.D[1];
    if ((rc = solver_setup(units, nunits, nd, o.krylov_dim, 1, tol1, require_cluster, o.keep, B64,
                           c.s)))
      return rc;
    if ((rc = solver_rq_refine(G, tiles, ntiles, units, nunits, ckey, B64,
                               (const float*)stage1_vec, c.s)))
      return rc;
    if ((rc = solver_write_vector(G, tiles, ntiles, units, ckey, B64, 0, 1, out, cand, 0, c.s)))
      return rc;
    trace_mark(c.s, "cand %d fp64 rayleigh quotient", cand);
    if (o.polish_cycles > 0) {
      // stage 3: at most polish_cycles FP64 Lanczos cycles of polish_dim steps,
      // started from the FP32 vector, stopping early at tol; a unit keeps the
      // polished vector only where it lowered the FP64 residual
      if ((rc = solver_setup(units, nunits, nd, o.polish_dim, o.polish_cycles, o.tol,
                             require_cluster, o.keep, B64, c.s)))
        return rc;
      if ((rc = solver_lanczos(G, tiles, ntiles, units, nunits, ckey, B64, 0, Mp, sd, nullptr,
                               (const float*)stage1_vec, use_graph, c.s)))
        return rc;
      if ((rc = solver_write_vector(G, tiles, ntiles, units, ckey, B64, 0, 0, out, cand, 1, c.s)))
        return rc;
      if ((rc = solver_keep_better(units, nunits, cand, tol1, c.s))) return rc;
      trace_mark(c.s, "cand %d fp64 polish (<= %d cycles of %d)", cand, o.polish_cycles, Mp);
    }
  }
  // statistics
  RSB_CK(cudaMemsetAsync(&cn->capped, 0, sizeof(int), c.s));
  RSB_CK(cudaMemsetAsync(&cn->resid_max, 0, sizeof(double), c.s));
  if ((rc = solver_stats(units, nunits, &cn->capped, &cn->resid_max, c.s))) return rc;
  Counters h;
  RSB_CK(cudaMemcpyAsync(&h, cn, sizeof(Counters), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  if (trace_on())
    fprintf(stderr, "[rsb]               cand %d: %lld cycles, %d capped, resid_max %.3e\n", cand,
            (long long)h.cycles, h.capped, h.resid_max);
  rs.solves += 1;
  rs.cycles += h.cycles;
  if (inverse) rs.inner += h.inner;
  rs.nonconv += h.capped;
  rs.resid_max = std::max(rs.resid_max, h.resid_max);
  return RSB_OK;
}

// All candidates, rotation, orientation, split and choice for the level's units.
static int split_units(Ctx& c, const LevelGraph& G, std::vector<Unit>& hunits,
                       const std::vector<Tile>& htiles, const rsb_options& o, RunStats& rs) {
  const int nunits = (int)hunits.size();
  const int ntiles = (int)htiles.size();
  if (nunits == 0) return RSB_OK;
  int rc;
  if ((rc = devbuf_reserve(c.units, sizeof(Unit) * nunits))) return rc;
  if ((rc = devbuf_reserve(c.tiles, sizeof(Tile) * ntiles))) return rc;
  if ((rc = devbuf_reserve(c.partials, 4 * sizeof(double) * (size_t)RSB_MAXC * ntiles + 64))) return rc;
  if ((rc = devbuf_reserve(c.hist, sizeof(int) * 256 * (size_t)nunits))) return rc;
  if ((rc = devbuf_reserve(c.mom, sizeof(double) * 24 * (size_t)nunits))) return rc;
  if ((rc = devbuf_reserve(c.sbuf, sizeof(double) * RSB_SSTRIDE * (size_t)nunits))) return rc;
  for (int k = 0; k < 3; ++k)
    if ((rc = devbuf_reserve(c.cand[k], sizeof(double) * (size_t)(G.n + 32)))) return rc;
  RSB_CK(cudaMemsetAsync(c.hist.p, 0, sizeof(int) * 256 * (size_t)nunits, c.s));
  Unit* units = dptr<Unit>(c.units);
  Tile* tiles = dptr<Tile>(c.tiles);
  RSB_CK(cudaMemcpyAsync(units, hunits.data(), sizeof(Unit) * nunits, cudaMemcpyHostToDevice, c.s));
  RSB_CK(cudaMemcpyAsync(tiles, htiles.data(), sizeof(Tile) * ntiles, cudaMemcpyHostToDevice, c.s));
  c.trmax = max_tile_rows(htiles);
  const uint64_t* ckey = dptr<uint64_t>(c.ckey);
  double* partials = dptr<double>(c.partials);
  int64_t maxn = 0;
  for (auto& u : hunits) maxn = std::max<int64_t>(maxn, u.n);
  if (o.method == RSB_RCB) {
    // recursive coordinate bisection: the unit's coordinate along its longest
    // extent takes the place of the Fiedler vector; lower coordinates go left
    double* v0 = dptr<double>(c.cand[0]);
    uint8_t* side = dptr<uint8_t>(c.side);
    int* hist = dptr<int>(c.hist);
    if ((rc = launch_rcb_vector(G, tiles, ntiles, units, dptr<double>(c.coords_cat), v0, partials,
                                c.s)) ||
        (rc = launch_orient(G, tiles, ntiles, units, ckey, v0, 0, o.tie_rel, partials, c.s, 1)) ||
        (rc = launch_select(G, tiles, ntiles, units, nunits, ckey, v0, 0, 0, hist, c.s)) ||
        (rc = launch_split_below(G, tiles, ntiles, units, ckey, v0, 0, partials, c.s)) ||
        (rc = launch_select(G, tiles, ntiles, units, nunits, ckey, v0, 1, 0, hist, c.s)) ||
        (rc = launch_split_assign(G, tiles, ntiles, units, ckey, v0, side, 0, c.s)))
      return rc;
    return RSB_OK;
  }
  if ((rc = launch_degree_max(G, tiles, ntiles, units, ckey, partials, c.s))) return rc;
  const int ncmax = o.degenerate_policy == RSB_DEGEN_RESOLVE ? 3 : 1;
  for (int cand = 0; cand < ncmax; ++cand) {
    if ((rc = solve_candidate(c, G, tiles, ntiles, units, nunits, maxn, o, cand, rs, hunits)))
      return rc;
    if (cand > 0 && (rc = solver_cluster_check(units, nunits, cand, o.cluster_tol, c.s))) return rc;
  }
  double* v0 = dptr<double>(c.cand[0]);
  double* v1 = dptr<double>(c.cand[1]);
  double* v2 = dptr<double>(c.cand[2]);
  if (ncmax > 1 &&
      (rc = solver_quartic(tiles, ntiles, units, nunits, ckey, v0, v1, v2, partials,
                           dptr<double>(c.mom), c.s)))
    return rc;
  uint8_t* side = dptr<uint8_t>(c.side);
  int* hist = dptr<int>(c.hist);
  double* vs[3] = {v0, v1, v2};
  for (int cand = 0; cand < ncmax; ++cand) {
    if ((rc = launch_orient(G, tiles, ntiles, units, ckey, vs[cand], cand, o.tie_rel, partials, c.s)))
      return rc;
    if ((rc = launch_select(G, tiles, ntiles, units, nunits, ckey, vs[cand], 0, cand, hist, c.s)))
      return rc;
    if ((rc = launch_split_below(G, tiles, ntiles, units, ckey, vs[cand], cand, partials, c.s)))
      return rc;
    if ((rc = launch_select(G, tiles, ntiles, units, nunits, ckey, vs[cand], 1, cand, hist, c.s)))
      return rc;
    if ((rc = launch_split_assign(G, tiles, ntiles, units, ckey, vs[cand], side, cand, c.s)))
      return rc;
  }
  if (ncmax > 1) {
    for (int cand = 0; cand < ncmax; ++cand)
      if ((rc = launch_cut(G, tiles, ntiles, units, ckey, side, cand, partials, c.s))) return rc;
    for (int cand = 1; cand < ncmax; ++cand)
      if ((rc = launch_choose(G, tiles, ntiles, units, ckey, side, cand, partials, c.s))) return rc;
  }
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// the level loop
// ----------------------------------------------------------------------------
struct MeshInfo {
  int64_t N;
  int32_t P;
};

static inline int64_t fl(int64_t p, int64_t N, int64_t P) { return (p * N) / P; }

// perm / iperm: the level-0 row order (see build_level0); home_out: where to
// copy the caller row of every row of the final level (the RCB reordering)
static int run_rsb(Ctx& c, const std::vector<MeshIn>& meshes, const std::vector<int32_t>& nparts,
                   const rsb_options& o, int32_t* part_concat, rsb_stats* st,
                   const int64_t* perm = nullptr, const int32_t* iperm = nullptr,
                   int64_t* home_out = nullptr) {
  LevelGraph G;
  trace_mark(c.s, "call start");
  int rc = build_level0(c, meshes, o.validate, G, perm, iperm);
  if (rc) return rc;
  const bool rcb = o.method == RSB_RCB;
  if (rcb) {
    int64_t nall = 0;
    for (auto& m : meshes) nall += m.n;
    if ((rc = devbuf_reserve(c.coords_cat, 3 * sizeof(double) * (size_t)(nall + 32)))) return rc;
    int64_t o3 = 0;
    for (auto& m : meshes) {
      if (!m.coords) return rsb_set_error(RSB_EINVAL, "coordinate bisection needs coords");
      RSB_CK(cudaMemcpyAsync(dptr<double>(c.coords_cat) + o3, m.coords, 3 * sizeof(double) * m.n,
                             cudaMemcpyDeviceToDevice, c.s));
      o3 += 3 * m.n;
    }
  }
  trace_mark(c.s, "level-0 ingest: %lld rows, %lld stored entries", (long long)G.n,
             (long long)G.nent);
  const int64_t N = G.n;
  std::vector<SegHost> segs;
  int64_t off = 0;
  for (size_t m = 0; m < meshes.size(); ++m) {
    SegHost s;
    s.row0 = off;
    s.n = meshes[m].n;
    s.p0 = 0;
    s.p1 = nparts[m];
    s.mesh = (int32_t)m;
    s.nleft = 0;
    segs.push_back(s);
    off += meshes[m].n;
  }
  if ((rc = devbuf_reserve(c.parent, sizeof(int32_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.cmin, sizeof(uint64_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.ckey, sizeof(uint64_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.side, sizeof(uint8_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.tmp64, sizeof(int64_t) * (N + 32)))) return rc;
  if ((rc = devbuf_reserve(c.newpos, sizeof(int64_t) * (N + 32)))) return rc;
  RunStats rs;
  int64_t bisected = 0;
  int levels = 0;
  double lambda_first = 0.0;
  int cur = 0;
  Counters* cn = dptr<Counters>(c.counters);
  for (int level = 0; level < 64; ++level) {
    const int nseg = (int)segs.size();
    bool any = false;
    for (auto& s : segs)
      if (s.p1 - s.p0 >= 2) any = true;
    if (!any) break;
    ++levels;
    trace_mark(c.s, "level %d start: %d segments, %lld rows", level, nseg, (long long)G.n);
    // R6 split sizes and the next level's segment table
    std::vector<SegHost> next;
    std::vector<int64_t> h_row0(nseg), h_nleft(nseg);
    std::vector<int32_t> h_child0(nseg);
    for (int i = 0; i < nseg; ++i) {
      SegHost& s = segs[i];
      h_row0[i] = s.row0;
      h_child0[i] = (int32_t)next.size();
      if (s.p1 - s.p0 >= 2) {
        const int64_t Nm = meshes[s.mesh].n, Pm = nparts[s.mesh];
        const int32_t pm = s.p0 + (s.p1 - s.p0) / 2;
        s.nleft = fl(pm, Nm, Pm) - fl(s.p0, Nm, Pm);
        bisected += s.n;
        SegHost L = {s.row0, s.nleft, s.p0, pm, s.mesh, 0};
        SegHost R = {s.row0 + s.nleft, s.n - s.nleft, pm, s.p1, s.mesh, 0};
        next.push_back(L);
        next.push_back(R);
      } else {
        s.nleft = s.n;
        next.push_back(s);
      }
      h_nleft[i] = s.nleft;
    }
    // components of every segment
    if ((rc = devbuf_reserve(c.seg_ncomp, sizeof(int32_t) * nseg))) return rc;
    std::vector<int32_t> ncomp(nseg, 1);
    if (rcb) {
      // geometric splits ignore connectivity: every segment is one piece
      RSB_CK(cudaMemsetAsync(c.ckey.p, 0, sizeof(uint64_t) * (size_t)G.n, c.s));
    } else {
      RSB_CK(cudaMemsetAsync(c.seg_ncomp.p, 0, sizeof(int32_t) * nseg, c.s));
      if ((rc = launch_cc(G, dptr<int32_t>(c.parent), dptr<uint64_t>(c.cmin), &cn->flag, c.s)))
        return rc;
      if ((rc = launch_cc_spread(G, dptr<int32_t>(c.parent), dptr<uint64_t>(c.cmin),
                                 dptr<uint64_t>(c.ckey), &cn->flag, c.s)))
        return rc;
      if ((rc = launch_comp_count(G, dptr<int32_t>(c.parent), dptr<int32_t>(c.seg_ncomp), c.s)))
        return rc;
      RSB_CK(cudaMemcpyAsync(ncomp.data(), c.seg_ncomp.p, sizeof(int32_t) * nseg,
                             cudaMemcpyDeviceToHost, c.s));
      RSB_CK(cudaStreamSynchronize(c.s));
    }
    // straddling component of segments that fell apart (radix select on the
    // component key with rank nleft)
    std::vector<uint64_t> keystar(nseg, 0);
    std::vector<int64_t> kbelow(nseg, 0), keq(nseg, 0);
    std::vector<uint8_t> split(nseg, 0);
    {
      std::vector<Unit> su;
      std::vector<int> su_seg;
      for (int i = 0; i < nseg; ++i) {
        if (segs[i].p1 - segs[i].p0 < 2) continue;
        split[i] = ncomp[i] > 1 ? 2 : 1;
        if (ncomp[i] <= 1) continue;
        Unit u = blank_unit();
        u.row0 = (int32_t)segs[i].row0;
        u.nrows = (int32_t)segs[i].n;
        u.seg = i;
        u.valid = 1;
        u.n = segs[i].n;
        u.k = segs[i].nleft;
        su.push_back(u);
        su_seg.push_back(i);
      }
      if (!su.empty()) {
        std::vector<Tile> st2;
        std::vector<int64_t> su_mesh;
        for (const Unit& u : su) su_mesh.push_back(meshes[segs[u.seg].mesh].n);
        make_tiles(su, st2, RSB_MINR, su_mesh);
        if ((rc = devbuf_reserve(c.sunits, sizeof(Unit) * su.size()))) return rc;
        if ((rc = devbuf_reserve(c.stiles, sizeof(Tile) * st2.size()))) return rc;
        if ((rc = devbuf_reserve(c.hist, sizeof(int) * 256 * su.size()))) return rc;
        RSB_CK(cudaMemsetAsync(c.hist.p, 0, sizeof(int) * 256 * su.size(), c.s));
        RSB_CK(cudaMemcpyAsync(c.sunits.p, su.data(), sizeof(Unit) * su.size(),
                               cudaMemcpyHostToDevice, c.s));
        RSB_CK(cudaMemcpyAsync(c.stiles.p, st2.data(), sizeof(Tile) * st2.size(),
                               cudaMemcpyHostToDevice, c.s));
        if ((rc = launch_select(G, dptr<Tile>(c.stiles), (int)st2.size(), dptr<Unit>(c.sunits),
                                (int)su.size(), dptr<uint64_t>(c.ckey), nullptr, 2, 0,
                                dptr<int>(c.hist), c.s)))
          return rc;
        RSB_CK(cudaMemcpyAsync(su.data(), c.sunits.p, sizeof(Unit) * su.size(),
                               cudaMemcpyDeviceToHost, c.s));
        RSB_CK(cudaStreamSynchronize(c.s));
        for (size_t q = 0; q < su.size(); ++q) {
          const int i = su_seg[q];
          keystar[i] = su[q].sel_prefix;
          kbelow[i] = su[q].sel_below;
          keq[i] = su[q].sel_eq;
        }
      }
    }
    // units: one Fiedler problem per bisected segment (or none when the
    // components fill the left part exactly)
    std::vector<Unit> hunits;
    std::vector<int32_t> seg_unit(nseg, -1);
    for (int i = 0; i < nseg; ++i) {
      if (!split[i]) continue;
      Unit u = blank_unit();
      u.row0 = (int32_t)segs[i].row0;
      u.nrows = (int32_t)segs[i].n;
      u.seg = i;
      u.valid = 1;
      if (split[i] == 1) {
        u.masked = 0;
        u.n = segs[i].n;
        u.k = segs[i].nleft;
      } else {
        if (kbelow[i] + keq[i] <= segs[i].nleft) continue;  // fits exactly
        u.masked = 1;
        u.key = keystar[i];
        u.n = keq[i];
        u.k = segs[i].nleft - kbelow[i];
      }
      u.isn = 1.0 / std::sqrt((double)u.n);
      seg_unit[i] = (int32_t)hunits.size();
      hunits.push_back(u);
    }
    std::vector<Tile> htiles;
    std::vector<int64_t> hmesh;
    for (const Unit& u : hunits) hmesh.push_back(meshes[segs[u.seg].mesh].n);
    make_tiles(hunits, htiles, o.tile_rows > 0 ? o.tile_rows : RSB_MINR, hmesh);
    trace_mark(c.s, "level %d components and units", level);
    if ((rc = split_units(c, G, hunits, htiles, o, rs))) return rc;
    trace_mark(c.s, "level %d split (%d units)", level, (int)hunits.size());
    if (level == 0 && !hunits.empty() && !rcb) {
      Unit u0;
      RSB_CK(cudaMemcpyAsync(&u0, dptr<Unit>(c.units), sizeof(Unit), cudaMemcpyDeviceToHost, c.s));
      RSB_CK(cudaStreamSynchronize(c.s));
      lambda_first = u0.lam[0];
    }
    // final side of every row, then compaction into the next level
    if ((rc = devbuf_reserve(c.seg_row0, sizeof(int64_t) * nseg))) return rc;
    if ((rc = devbuf_reserve(c.seg_nleft, sizeof(int64_t) * nseg))) return rc;
    if ((rc = devbuf_reserve(c.seg_child0, sizeof(int32_t) * nseg))) return rc;
    if ((rc = devbuf_reserve(c.seg_split, sizeof(uint8_t) * nseg))) return rc;
    if ((rc = devbuf_reserve(c.seg_keystar, sizeof(uint64_t) * nseg))) return rc;
    if ((rc = devbuf_reserve(c.seg_unit, sizeof(int32_t) * nseg))) return rc;
    // connected segments: every row has the same key, use the unit's side
    std::vector<uint64_t> ks(nseg);
    std::vector<uint8_t> spl(nseg);
    for (int i = 0; i < nseg; ++i) {
      spl[i] = split[i] ? 1 : 0;
      ks[i] = split[i] == 2 ? keystar[i] : 0;
    }
    RSB_CK(cudaMemcpyAsync(c.seg_row0.p, h_row0.data(), sizeof(int64_t) * nseg,
                           cudaMemcpyHostToDevice, c.s));
    RSB_CK(cudaMemcpyAsync(c.seg_nleft.p, h_nleft.data(), sizeof(int64_t) * nseg,
                           cudaMemcpyHostToDevice, c.s));
    RSB_CK(cudaMemcpyAsync(c.seg_child0.p, h_child0.data(), sizeof(int32_t) * nseg,
                           cudaMemcpyHostToDevice, c.s));
    RSB_CK(cudaMemcpyAsync(c.seg_split.p, spl.data(), nseg, cudaMemcpyHostToDevice, c.s));
    RSB_CK(cudaMemcpyAsync(c.seg_unit.p, seg_unit.data(), sizeof(int32_t) * nseg,
                           cudaMemcpyHostToDevice, c.s));
    // for connected segments the comparison key must equal every row's key:
    // give them the key of the segment's first row
    RSB_CK(cudaMemcpyAsync(c.seg_keystar.p, ks.data(), sizeof(uint64_t) * nseg,
                           cudaMemcpyHostToDevice, c.s));
    for (int i = 0; i < nseg; ++i)
      if (split[i] == 1)
        RSB_CK(cudaMemcpyAsync(dptr<uint64_t>(c.seg_keystar) + i, dptr<uint64_t>(c.ckey) + segs[i].row0,
                               sizeof(uint64_t), cudaMemcpyDeviceToDevice, c.s));
    if ((rc = launch_finalize_side(G, dptr<uint8_t>(c.seg_split), dptr<uint64_t>(c.seg_keystar),
                                   dptr<int32_t>(c.seg_unit), dptr<Unit>(c.units),
                                   dptr<uint64_t>(c.ckey), dptr<uint8_t>(c.side), c.s)))
      return rc;
    LevelGraph H;
    const int nxt = cur ^ 1;
    H.slice_ptr = dptr<int64_t>(c.slice_ptr[nxt]);
    H.deg = dptr<int32_t>(c.deg[nxt]);
    H.gid = dptr<int64_t>(c.gid[nxt]);
    H.home = dptr<int64_t>(c.home[nxt]);
    H.row_seg = dptr<int32_t>(c.row_seg[nxt]);
    if ((rc = launch_compact(G, H, dptr<uint8_t>(c.side), dptr<int64_t>(c.seg_row0),
                             dptr<int64_t>(c.seg_nleft), dptr<int32_t>(c.seg_child0), nseg,
                             dptr<int64_t>(c.newpos), dptr<int64_t>(c.tmp64), dptr<int32_t>(c.len),
                             dptr<int64_t>(c.slice_sz), c.scan_tmp.p, c.scan_tmp.cap, c.ent[nxt],
                             c.s)))
      return rc;
    trace_mark(c.s, "level %d compaction", level);
    G = H;
    cur = nxt;
    segs.swap(next);
  }
  // part ids
  const int nseg = (int)segs.size();
  std::vector<int32_t> p0(nseg);
  for (int i = 0; i < nseg; ++i) p0[i] = segs[i].p0;
  if ((rc = devbuf_reserve(c.seg_child0, sizeof(int32_t) * nseg))) return rc;
  RSB_CK(cudaMemcpyAsync(c.seg_child0.p, p0.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice,
                         c.s));
  if ((rc = launch_write_parts(G, dptr<int32_t>(c.seg_child0), part_concat, c.s))) return rc;
  if (home_out)
    RSB_CK(cudaMemcpyAsync(home_out, G.home, sizeof(int64_t) * (size_t)G.n,
                           cudaMemcpyDeviceToDevice, c.s));
  // CC error flag (a bound that can never be reached in a correct run)
  RSB_CK(cudaMemcpyAsync(c.h_pinned, &cn->flag, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  if (c.h_pinned[0] & 32) return rsb_set_error(RSB_ETIMEOUT, "union-find bound reached");
  if (st) {
    st->levels = levels;
    st->nonconverged = rs.nonconv;
    st->solves = rs.solves;
    st->cycles = rs.cycles;
    st->inner = rs.inner;
    st->elements_bisected = bisected;
    st->lambda_first = lambda_first;
    st->resid_max = rs.resid_max;
  }
  return rs.nonconv ? RSB_ENOCONV : RSB_OK;
}

// ----------------------------------------------------------------------------
// ABI
// ----------------------------------------------------------------------------
static int begin_call(Ctx** pc, void* stream) {
  int rc = ctx_get(pc);
  if (rc) return rc;
  Ctx& c = **pc;
  RSB_CK(cudaEventRecord(c.ev_in, (cudaStream_t)stream));
  RSB_CK(cudaStreamWaitEvent(c.s, c.ev_in, 0));
  return RSB_OK;
}

static int end_call(Ctx& c, void* stream, int rc) {
  cudaError_t e1 = cudaEventRecord(c.ev_out, c.s);
  cudaError_t e2 = cudaStreamWaitEvent((cudaStream_t)stream, c.ev_out, 0);
  cudaError_t e3 = cudaStreamSynchronize(c.s);
  stage_clear(c);
  if (rc) return rc;
  if (e1 != cudaSuccess) return rsb_set_cuda_error(e1, "cudaEventRecord");
  if (e2 != cudaSuccess) return rsb_set_cuda_error(e2, "cudaStreamWaitEvent");
  if (e3 != cudaSuccess) return rsb_set_cuda_error(e3, "cudaStreamSynchronize");
  return RSB_OK;
}

static int mesh_from(Ctx& c, const rsb_csr* g, MeshIn& m) {
  if (!g) return rsb_set_error(RSB_EINVAL, "NULL graph");
  if (g->n < 0 || g->n >= RSB_MAXN) return rsb_set_error(RSB_EINVAL, "n out of range");
  if (g->n > 0 && (!g->row_ptr || (!g->col && false)))
    return rsb_set_error(RSB_EINVAL, "NULL row_ptr");
  m.n = g->n;
  int64_t nnz = 0;
  if (g->n > 0) {
    if (is_device_ptr(g->row_ptr)) {
      RSB_CK(cudaMemcpy(&nnz, g->row_ptr + g->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
      nnz = g->row_ptr[g->n];
    }
  }
  if (nnz < 0) return rsb_set_error(RSB_EINVAL, "row_ptr[n] < 0");
  if (nnz > 0 && !g->col) return rsb_set_error(RSB_EINVAL, "NULL col");
  m.nnz = nnz;
  int rc;
  if ((rc = stage_in(c, g->row_ptr, (size_t)(g->n + 1), &m.row_ptr))) return rc;
  if ((rc = stage_in(c, g->col, (size_t)nnz, &m.col))) return rc;
  if ((rc = stage_in(c, g->weight, (size_t)nnz, &m.wt))) return rc;
  if ((rc = stage_in(c, g->gid, (size_t)g->n, &m.gid))) return rc;
  if ((rc = stage_in(c, g->coords, (size_t)(3 * g->n), &m.coords))) return rc;
  return RSB_OK;
}

__global__ void k_make_perm(const int64_t* __restrict__ home, int64_t n, int64_t off, int64_t* perm,
                            int32_t* iperm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p = home[off + i] - off;
  perm[off + i] = p;
  iperm[off + p] = (int32_t)i;
}

// The RCB order of every mesh: RCB into 2^k leaves of 512..1023 elements; the
// rows of the final level, in order, are the new row order.
static int rcb_order(Ctx& c, const std::vector<MeshIn>& meshes, const rsb_options& o,
                     const int64_t** perm, const int32_t** iperm) {
  int64_t N = 0;
  std::vector<int32_t> leaves;
  for (auto& m : meshes) {
    if (!m.coords) return rsb_set_error(RSB_EINVAL, "reorder needs coords for every mesh");
    int32_t p = 1;
    while ((int64_t)p * 2 * 512 <= m.n) p *= 2;
    leaves.push_back(p);
    N += m.n;
  }
  int rc;
  if ((rc = devbuf_reserve(c.perm, sizeof(int64_t) * (size_t)(N + 32))) ||
      (rc = devbuf_reserve(c.iperm, sizeof(int32_t) * (size_t)(N + 32))) ||
      (rc = devbuf_reserve(c.rcb_home, sizeof(int64_t) * (size_t)(N + 32))))
    return rc;
  rsb_options orcb = o;
  orcb.method = RSB_RCB;
  orcb.batched = 1;
  if ((rc = run_rsb(c, meshes, leaves, orcb, dptr<int32_t>(c.part_concat), nullptr, nullptr,
                    nullptr, dptr<int64_t>(c.rcb_home))))
    return rc;
  int64_t off = 0;
  for (auto& m : meshes) {
    if (m.n > 0) {
      k_make_perm<<<(unsigned)((m.n + RSB_BLOCK - 1) / RSB_BLOCK), RSB_BLOCK, 0, c.s>>>(
          dptr<int64_t>(c.rcb_home), m.n, off, dptr<int64_t>(c.perm), dptr<int32_t>(c.iperm));
      RSB_CKL("k_make_perm");
    }
    off += m.n;
  }
  trace_mark(c.s, "RCB reordering of %lld elements", (long long)N);
  *perm = dptr<int64_t>(c.perm);
  *iperm = dptr<int32_t>(c.iperm);
  return RSB_OK;
}

extern "C" int rsb_partition_batch(const rsb_csr* gs, int32_t nmesh, const int32_t* nparts,
                                   const rsb_options* opt, int32_t* const* parts, rsb_stats* st,
                                   void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  g_launches = 0;
  if (!gs || nmesh < 1 || !nparts || !parts) return rsb_set_error(RSB_EINVAL, "batch arguments");
  rsb_options o;
  rsb_options_default(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  for (int m = 0; m < nmesh; ++m) {
    if (gs[m].n < 1 || nparts[m] < 1 || nparts[m] > gs[m].n)
      return rsb_set_error(RSB_EINVAL, "need 1 <= nparts <= n for every mesh");
    if (!parts[m]) return rsb_set_error(RSB_EINVAL, "NULL part output");
  }
  Ctx* pc = nullptr;
  rc = begin_call(&pc, stream);
  if (rc) return rc;
  Ctx& c = *pc;
  std::vector<MeshIn> meshes(nmesh);
  std::vector<int32_t> np(nparts, nparts + nmesh);
  int64_t N = 0;
  for (int m = 0; m < nmesh; ++m) {
    rc = mesh_from(c, &gs[m], meshes[m]);
    if (rc) return end_call(c, stream, rc);
    N += meshes[m].n;
  }
  if (N >= RSB_MAXN) return end_call(c, stream, rsb_set_error(RSB_EINVAL, "too many rows"));
  rc = devbuf_reserve(c.part_concat, sizeof(int32_t) * (N + 32));
  const int64_t* perm = nullptr;
  const int32_t* iperm = nullptr;
  if (!rc && o.reorder && o.method != RSB_RCB) {
    // locality reordering: recursive coordinate bisection of every mesh into
    // leaves of 512 to 1023 elements; the spectral recursion then starts from
    // the elements in RCB order (the part ids still land in caller order)
    rc = rcb_order(c, meshes, o, &perm, &iperm);
  }
  if (!rc) {
    if (o.batched) {
      rc = run_rsb(c, meshes, np, o, dptr<int32_t>(c.part_concat), st, perm, iperm);
    } else {
      // one mesh at a time; statistics summed
      rsb_stats acc;
      memset(&acc, 0, sizeof(acc));
      int64_t off = 0;
      for (int m = 0; m < nmesh && (rc == RSB_OK || rc == RSB_ENOCONV); ++m) {
        rsb_stats one;
        memset(&one, 0, sizeof(one));
        std::vector<MeshIn> single(1, meshes[m]);
        std::vector<int32_t> p1(1, np[m]);
        const int r1 = run_rsb(c, single, p1, o, dptr<int32_t>(c.part_concat) + off, &one,
                               perm ? perm + off : nullptr, iperm ? iperm + off : nullptr);
        if (r1 && r1 != RSB_ENOCONV) { rc = r1; break; }
        if (r1 == RSB_ENOCONV) rc = RSB_ENOCONV;
        acc.levels = std::max(acc.levels, one.levels);
        acc.nonconverged += one.nonconverged;
        acc.solves += one.solves;
        acc.cycles += one.cycles;
        acc.inner += one.inner;
        acc.elements_bisected += one.elements_bisected;
        if (m == 0) acc.lambda_first = one.lambda_first;
        acc.resid_max = std::max(acc.resid_max, one.resid_max);
        off += meshes[m].n;
      }
      if (st) *st = acc;
    }
  }
  if (rc == RSB_OK || rc == RSB_ENOCONV) {
    int64_t off = 0;
    for (int m = 0; m < nmesh; ++m) {
      cudaError_t e = cudaMemcpyAsync(parts[m], dptr<int32_t>(c.part_concat) + off,
                                      sizeof(int32_t) * meshes[m].n, cudaMemcpyDefault, c.s);
      if (e != cudaSuccess) {
        rc = rsb_set_cuda_error(e, "copy of part ids");
        break;
      }
      off += meshes[m].n;
    }
  }
  rc = end_call(c, stream, rc);
  if (st) {
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st->kernel_launches = g_launches;
  }
  return rc;
}

extern "C" int rsb_partition(const rsb_csr* g, int32_t nparts, const rsb_options* o,
                             int32_t* part, rsb_stats* st, void* stream) {
  if (!g) return rsb_set_error(RSB_EINVAL, "NULL graph");
  int32_t* const parts[1] = {part};
  return rsb_partition_batch(g, 1, &nparts, o, parts, st, stream);
}

// ----------------------------------------------------------------------------
// rsb_autotune: tile rows x launch mode, timed on the caller's workload
// ----------------------------------------------------------------------------
static const int kTuneTile[RSB_TUNE_CANDIDATES] = {2, 4, 8, 2, 4, 8};
static const int kTuneLaunch[RSB_TUNE_CANDIDATES] = {3, 3, 3, 1, 1, 1};

extern "C" int rsb_autotune(const rsb_csr* gs, int32_t nmesh, const int32_t* nparts,
                            rsb_options* o, int32_t* const* parts, double* ms_out,
                            void* stream) {
  if (!gs || !nparts || !o || !parts || nmesh < 1) return rsb_set_error(RSB_EINVAL, "autotune args");
  int rc = check_options(*o);
  if (rc) return rc;
  // one bisection level, two Lanczos cycles, no polish and no deflated
  // candidates: the kernels and launches of a cycle, at the workload's size
  std::vector<int32_t> np(nmesh);
  for (int m = 0; m < nmesh; ++m) np[m] = std::min<int32_t>(nparts[m], 2);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RSB_CK(cudaEventCreate(&e0));
  RSB_CK(cudaEventCreate(&e1));
  double best = 1e300;
  int pick = 0;
  for (int c = 0; c < RSB_TUNE_CANDIDATES && rc == RSB_OK; ++c) {
    rsb_options t = *o;
    t.tile_rows = kTuneTile[c];
    t.use_graph = kTuneLaunch[c];
    t.max_restarts = 2;
    t.tol = 1e-300;
    t.mixed_tol = 1e-300;
    t.polish_cycles = 0;
    t.degenerate_policy = RSB_DEGEN_NONE;
    t.method = RSB_LANCZOS;
    double ms = 1e300;
    for (int rep = 0; rep < 3 && rc == RSB_OK; ++rep) {  // first call warms up
      cudaEventRecord(e0, s);
      int r = rsb_partition_batch(gs, nmesh, np.data(), &t, parts, nullptr, stream);
      cudaEventRecord(e1, s);
      if (r != RSB_OK && r != RSB_ENOCONV) {
        rc = r;
        break;
      }
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        rc = rsb_set_cuda_error(ce, "autotune timing");
        break;
      }
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      if (rep > 0) ms = std::min(ms, (double)f);
    }
    if (ms_out) ms_out[c] = ms;
    if (rc == RSB_OK && ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  o->tile_rows = kTuneTile[pick];
  o->use_graph = kTuneLaunch[pick];
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// rsb_fiedler
// ----------------------------------------------------------------------------
__global__ void k_fiedler_out(const double* __restrict__ v, int32_t n, const Unit* u,
                              double* out) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r < n) out[r] = u->sign * v[r];
}

extern "C" int rsb_fiedler(const rsb_csr* g, const rsb_options* opt, double* lambda2, double* v,
                           double* resid, void* stream) {
  g_launches = 0;
  if (!g || !lambda2 || !v) return rsb_set_error(RSB_EINVAL, "fiedler arguments");
  if (g->n < 2) return rsb_set_error(RSB_EINVAL, "rsb_fiedler needs n >= 2");
  rsb_options o;
  rsb_options_default(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  if (o.method == RSB_RCB) return rsb_set_error(RSB_EINVAL, "rsb_fiedler needs a spectral method");
  Ctx* pc = nullptr;
  rc = begin_call(&pc, stream);
  if (rc) return rc;
  Ctx& c = *pc;
  std::vector<MeshIn> meshes(1);
  rc = mesh_from(c, g, meshes[0]);
  if (rc) return end_call(c, stream, rc);
  LevelGraph G;
  rc = build_level0(c, meshes, o.validate, G);
  if (rc) return end_call(c, stream, rc);
  const int64_t N = G.n;
  if ((rc = devbuf_reserve(c.parent, sizeof(int32_t) * (N + 32))) ||
      (rc = devbuf_reserve(c.cmin, sizeof(uint64_t) * (N + 32))) ||
      (rc = devbuf_reserve(c.ckey, sizeof(uint64_t) * (N + 32))) ||
      (rc = devbuf_reserve(c.side, sizeof(uint8_t) * (N + 32))) ||
      (rc = devbuf_reserve(c.seg_ncomp, sizeof(int32_t) * 4)))
    return end_call(c, stream, rc);
  Counters* cn = dptr<Counters>(c.counters);
  RSB_CK(cudaMemsetAsync(c.seg_ncomp.p, 0, sizeof(int32_t), c.s));
  if ((rc = launch_cc(G, dptr<int32_t>(c.parent), dptr<uint64_t>(c.cmin), &cn->flag, c.s)) ||
      (rc = launch_cc_spread(G, dptr<int32_t>(c.parent), dptr<uint64_t>(c.cmin),
                             dptr<uint64_t>(c.ckey), &cn->flag, c.s)) ||
      (rc = launch_comp_count(G, dptr<int32_t>(c.parent), dptr<int32_t>(c.seg_ncomp), c.s)))
    return end_call(c, stream, rc);
  int ncomp = 0;
  RSB_CK(cudaMemcpyAsync(&ncomp, c.seg_ncomp.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  const bool v_dev = is_device_ptr(v);
  if (ncomp > 1) {
    // contrast vector of the component holding the smallest gid
    std::vector<uint64_t> key(N);
    std::vector<int64_t> gid(N);
    RSB_CK(cudaMemcpy(key.data(), c.ckey.p, sizeof(uint64_t) * N, cudaMemcpyDeviceToHost));
    RSB_CK(cudaMemcpy(gid.data(), G.gid, sizeof(int64_t) * N, cudaMemcpyDeviceToHost));
    uint64_t k0 = ~0ull;
    for (int64_t i = 0; i < N; ++i) k0 = std::min<uint64_t>(k0, key[i]);
    int64_t n1 = 0;
    for (int64_t i = 0; i < N; ++i) n1 += key[i] == k0;
    std::vector<double> h(N);
    double nrm = 0;
    for (int64_t i = 0; i < N; ++i) {
      h[i] = key[i] == k0 ? 1.0 / n1 : -1.0 / (N - n1);
      nrm += h[i] * h[i];
    }
    nrm = 1.0 / std::sqrt(nrm);
    double amax = 0;
    for (int64_t i = 0; i < N; ++i) {
      h[i] *= nrm;
      amax = std::max(amax, std::fabs(h[i]));
    }
    int64_t gs = -1;
    double gv = 0;
    for (int64_t i = 0; i < N; ++i)
      if (std::fabs(h[i]) >= 0.5 * amax && (gs < 0 || gid[i] < gs)) { gs = gid[i]; gv = h[i]; }
    if (gv > 0)
      for (auto& x : h) x = -x;
    RSB_CK(cudaMemcpy(v, h.data(), sizeof(double) * N, cudaMemcpyDefault));
    *lambda2 = 0.0;
    if (resid) *resid = 0.0;
    return end_call(c, stream, RSB_EDISCONNECTED);
  }
  std::vector<Unit> hunits(1, blank_unit());
  Unit& u = hunits[0];
  u.row0 = 0;
  u.nrows = (int32_t)N;
  u.valid = 1;
  u.n = N;
  u.k = N / 2;
  u.isn = 1.0 / std::sqrt((double)N);
  std::vector<Tile> htiles;
  make_tiles(hunits, htiles, o.tile_rows > 0 ? o.tile_rows : RSB_MINR);
  c.trmax = max_tile_rows(htiles);
  const int ntiles = (int)htiles.size();
  if ((rc = devbuf_reserve(c.units, sizeof(Unit))) ||
      (rc = devbuf_reserve(c.tiles, sizeof(Tile) * ntiles)) ||
      (rc = devbuf_reserve(c.partials, 4 * sizeof(double) * (size_t)RSB_MAXC * ntiles + 64)) ||
      (rc = devbuf_reserve(c.sbuf, sizeof(double) * RSB_SSTRIDE)) ||
      (rc = devbuf_reserve(c.cand[0], sizeof(double) * (N + 32))))
    return end_call(c, stream, rc);
  RSB_CK(cudaMemcpyAsync(c.units.p, hunits.data(), sizeof(Unit), cudaMemcpyHostToDevice, c.s));
  RSB_CK(cudaMemcpyAsync(c.tiles.p, htiles.data(), sizeof(Tile) * ntiles, cudaMemcpyHostToDevice,
                         c.s));
  Unit* units = dptr<Unit>(c.units);
  Tile* tiles = dptr<Tile>(c.tiles);
  double* partials = dptr<double>(c.partials);
  if ((rc = launch_degree_max(G, tiles, ntiles, units, dptr<uint64_t>(c.ckey), partials, c.s)))
    return end_call(c, stream, rc);
  RunStats rs;
  if ((rc = solve_candidate(c, G, tiles, ntiles, units, 1, N, o, 0, rs, hunits)))
    return end_call(c, stream, rc);
  if ((rc = launch_orient(G, tiles, ntiles, units, dptr<uint64_t>(c.ckey), dptr<double>(c.cand[0]),
                          0, o.tie_rel, partials, c.s)))
    return end_call(c, stream, rc);
  double* vout = v;
  DevBuf tmpv;
  if (!v_dev) {
    if ((rc = devbuf_reserve(tmpv, sizeof(double) * N))) return end_call(c, stream, rc);
    vout = (double*)tmpv.p;
  }
  k_fiedler_out<<<(unsigned)((N + RSB_BLOCK - 1) / RSB_BLOCK), RSB_BLOCK, 0, c.s>>>(
      dptr<double>(c.cand[0]), (int32_t)N, units, vout);
  rsb_count_launch();
  RSB_CK(cudaGetLastError());
  if (!v_dev) RSB_CK(cudaMemcpyAsync(v, vout, sizeof(double) * N, cudaMemcpyDeviceToHost, c.s));
  Unit hu;
  RSB_CK(cudaMemcpyAsync(&hu, units, sizeof(Unit), cudaMemcpyDeviceToHost, c.s));
  rc = end_call(c, stream, rs.nonconv ? RSB_ENOCONV : RSB_OK);
  free_buf(tmpv);
  *lambda2 = hu.lam[0];
  if (resid) *resid = hu.res[0];
  return rc;
}

// ----------------------------------------------------------------------------
// Laplacian action and its bandwidth benchmark
// ----------------------------------------------------------------------------
static int lap_common(const rsb_csr* g, const void* x, void* y, int f32, int reps, double* ms,
                      double* bytes, void* stream) {
  if (!g || g->n < 1) return rsb_set_error(RSB_EINVAL, "graph");
  Ctx* pc = nullptr;
  int rc = begin_call(&pc, stream);
  if (rc) return rc;
  Ctx& c = *pc;
  std::vector<MeshIn> meshes(1);
  rc = mesh_from(c, g, meshes[0]);
  if (rc) return end_call(c, stream, rc);
  LevelGraph G;
  rc = build_level0(c, meshes, 0, G);
  if (rc) return end_call(c, stream, rc);
  const int64_t N = G.n;
  const size_t es = f32 ? 4 : 8;
  const void* xd = x;
  void* yd = y;
  DevBuf tx, ty;
  const bool xh = x && !is_device_ptr(x), yh = y && !is_device_ptr(y);
  if (reps > 0) {
    if ((rc = devbuf_reserve(tx, es * N)) || (rc = devbuf_reserve(ty, es * N)))
      return end_call(c, stream, rc);
    RSB_CK(cudaMemsetAsync(tx.p, 0, es * N, c.s));
    xd = tx.p;
    yd = ty.p;
  } else {
    if (xh) {
      if ((rc = devbuf_reserve(tx, es * N))) return end_call(c, stream, rc);
      RSB_CK(cudaMemcpyAsync(tx.p, x, es * N, cudaMemcpyHostToDevice, c.s));
      xd = tx.p;
    }
    if (yh) {
      if ((rc = devbuf_reserve(ty, es * N))) return end_call(c, stream, rc);
      yd = ty.p;
    }
  }
  auto apply = [&]() -> int {
    return f32 ? launch_spmv_f32(G, (const float*)xd, (float*)yd, c.s)
               : launch_spmv_f64(G, (const double*)xd, (double*)yd, c.s);
  };
  if (reps <= 0) {
    rc = apply();
    if (!rc && yh) {
      cudaError_t e = cudaMemcpyAsync(y, yd, es * N, cudaMemcpyDeviceToHost, c.s);
      if (e != cudaSuccess) rc = rsb_set_cuda_error(e, "copy y");
    }
  } else {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int w = 0; w < 3 && !rc; ++w) rc = apply();
    cudaEventRecord(e0, c.s);
    for (int i = 0; i < reps && !rc; ++i) rc = apply();
    cudaEventRecord(e1, c.s);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms) *ms = (double)t / reps;
    if (bytes) {
      int64_t nnz = meshes[0].nnz;
      *bytes = 4.0 * (double)nnz + 2.0 * (double)es * (double)N;
    }
  }
  rc = end_call(c, stream, rc);
  free_buf(tx);
  free_buf(ty);
  return rc;
}

extern "C" int rsb_laplacian_apply(const rsb_csr* g, const double* x, double* y, void* stream) {
  if (!x || !y) return rsb_set_error(RSB_EINVAL, "NULL vector");
  return lap_common(g, x, y, 0, 0, nullptr, nullptr, stream);
}
extern "C" int rsb_laplacian_apply_f32(const rsb_csr* g, const float* x, float* y, void* stream) {
  if (!x || !y) return rsb_set_error(RSB_EINVAL, "NULL vector");
  return lap_common(g, x, y, 1, 0, nullptr, nullptr, stream);
}
extern "C" int rsb_laplacian_bench(const rsb_csr* g, int f32, int reps, double* ms_per_apply,
                                   double* useful_bytes, void* stream) {
  if (reps < 1) return rsb_set_error(RSB_EINVAL, "reps");
  return lap_common(g, nullptr, nullptr, f32 ? 1 : 0, reps, ms_per_apply, useful_bytes, stream);
}

extern "C" void rsb_test_poison_barrier(int on) { g_rsb_poison_barrier = on ? 1 : 0; }

// ----------------------------------------------------------------------------
// element -> vertex ids: the dual graph and the matrix-free Laplacian (§5)
// ----------------------------------------------------------------------------
int gs_vertex_count(const int64_t* ev, int64_t cnt, unsigned long long* d_vmax, int* d_flag,
                    int64_t* V, cudaStream_t s);
int gs_buckets(const int64_t* ev, int64_t ne, int nv, int64_t V, int64_t* count, int64_t* cursor,
               int64_t* bptr, int32_t* bucket, int32_t* ev32, void* scan_tmp, size_t scan_bytes,
               cudaStream_t s);
int gs_row_lengths(int64_t ne, int nv, const int32_t* ev32, const int64_t* bptr,
                   const int32_t* bucket, int64_t* len, int* d_flag, cudaStream_t s);
int gs_fill_dual(int64_t ne, int nv, const int32_t* ev32, const int64_t* bptr,
                 const int32_t* bucket, const int64_t* row_ptr, int32_t* col, int32_t* wt,
                 cudaStream_t s);
int gs_apply(int f32, int64_t ne, int nv, int64_t V, const int32_t* ev32, const int64_t* bptr,
             const int32_t* bucket, const void* x, void* w, void* y, cudaStream_t s);

// Buckets of the elements at every vertex in the context's workspace; *V out.
static int gs_setup(Ctx& c, int64_t ne, int nv, const int64_t* ev_in, int64_t* V) {
  if (ne < 1 || ne >= RSB_MAXN || nv < 1 || nv > 8 || !ev_in)
    return rsb_set_error(RSB_EINVAL, "need 1 <= ne < 2^29, 1 <= nv <= 8 and vertex ids");
  const int64_t* ev = nullptr;
  int rc = stage_in(c, ev_in, (size_t)(ne * nv), &ev);
  if (rc) return rc;
  if ((rc = devbuf_reserve(c.gs_misc, 256))) return rc;
  unsigned long long* d_vmax = dptr<unsigned long long>(c.gs_misc);
  int* d_flag = (int*)(d_vmax + 1);
  if ((rc = gs_vertex_count(ev, ne * nv, d_vmax, d_flag, V, c.s))) return rc;
  const int64_t nV = *V;
  const size_t scan_bytes = scan_tmp_bytes(std::max<int64_t>(nV, ne) + 2);
  if ((rc = devbuf_reserve(c.gs_count, sizeof(int64_t) * (size_t)(nV + 2))) ||
      (rc = devbuf_reserve(c.gs_cursor, sizeof(int64_t) * (size_t)(nV + 2))) ||
      (rc = devbuf_reserve(c.gs_bptr, sizeof(int64_t) * (size_t)(nV + 2))) ||
      (rc = devbuf_reserve(c.gs_bucket, sizeof(int32_t) * (size_t)(ne * nv))) ||
      (rc = devbuf_reserve(c.gs_ev32, sizeof(int32_t) * (size_t)(ne * nv))) ||
      (rc = devbuf_reserve(c.scan_tmp, scan_bytes)))
    return rc;
  return gs_buckets(ev, ne, nv, nV, dptr<int64_t>(c.gs_count), dptr<int64_t>(c.gs_cursor),
                    dptr<int64_t>(c.gs_bptr), dptr<int32_t>(c.gs_bucket),
                    dptr<int32_t>(c.gs_ev32), c.scan_tmp.p, c.scan_tmp.cap, c.s);
}

extern "C" int rsb_dual_graph(int64_t ne, int nv, const int64_t* ev, int64_t* row_ptr,
                              int32_t* col, int32_t* weight, int64_t cap, int64_t* nnz,
                              void* stream) {
  if (!row_ptr || !nnz) return rsb_set_error(RSB_EINVAL, "row_ptr and nnz are needed");
  Ctx* pc = nullptr;
  int rc = begin_call(&pc, stream);
  if (rc) return rc;
  Ctx& c = *pc;
  int64_t V = 0;
  if ((rc = gs_setup(c, ne, nv, ev, &V))) return end_call(c, stream, rc);
  int* d_flag = (int*)(dptr<unsigned long long>(c.gs_misc) + 1);
  if ((rc = devbuf_reserve(c.gs_len, sizeof(int64_t) * (size_t)(ne + 2))) ||
      (rc = devbuf_reserve(c.gs_rowptr, sizeof(int64_t) * (size_t)(ne + 2))))
    return end_call(c, stream, rc);
  int64_t* len = dptr<int64_t>(c.gs_len);
  int64_t* rp = dptr<int64_t>(c.gs_rowptr);
  const int32_t* ev32 = dptr<int32_t>(c.gs_ev32);
  const int64_t* bptr = dptr<int64_t>(c.gs_bptr);
  const int32_t* bucket = dptr<int32_t>(c.gs_bucket);
  if ((rc = gs_row_lengths(ne, nv, ev32, bptr, bucket, len, d_flag, c.s)))
    return end_call(c, stream, rc);
  RSB_CK(cudaMemsetAsync(len + ne, 0, sizeof(int64_t), c.s));
  if ((rc = launch_scan_i64(len, rp, ne + 1, c.scan_tmp.p, c.scan_tmp.cap, c.s)))
    return end_call(c, stream, rc);
  int64_t total = 0;
  int flag = 0;
  RSB_CK(cudaMemcpyAsync(&total, rp + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RSB_CK(cudaStreamSynchronize(c.s));
  if (flag & 2)
    return end_call(c, stream, rsb_set_error(RSB_EINVAL, "an element meets more than 256 "
                                                         "other elements at its vertices"));
  if (flag & 4)
    return end_call(c, stream, rsb_set_error(RSB_EINVAL, "two elements share more than 7 "
                                                         "vertices (duplicate elements)"));
  *nnz = total;
  RSB_CK(cudaMemcpyAsync(row_ptr, rp, sizeof(int64_t) * (size_t)(ne + 1), cudaMemcpyDefault, c.s));
  if (col || weight) {
    if (!col || !weight || cap < total)
      return end_call(c, stream, rsb_set_error(RSB_EINVAL, "col and weight need room for nnz "
                                                           "entries (cap < nnz)"));
    const bool cd = is_device_ptr(col), wd = is_device_ptr(weight);
    DevBuf tc, tw;
    int32_t* colp = col;
    int32_t* wtp = weight;
    if (!cd && (rc = devbuf_reserve(tc, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1))))
      return end_call(c, stream, rc);
    if (!wd && (rc = devbuf_reserve(tw, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1)))) {
      free_buf(tc);
      return end_call(c, stream, rc);
    }
    if (!cd) colp = (int32_t*)tc.p;
    if (!wd) wtp = (int32_t*)tw.p;
    rc = gs_fill_dual(ne, nv, ev32, bptr, bucket, rp, colp, wtp, c.s);
    if (!rc && !cd)
      if (cudaMemcpyAsync(col, colp, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, c.s))
        rc = rsb_set_error(RSB_ECUDA, "copy col");
    if (!rc && !wd)
      if (cudaMemcpyAsync(weight, wtp, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, c.s))
        rc = rsb_set_error(RSB_ECUDA, "copy weight");
    rc = end_call(c, stream, rc);
    free_buf(tc);
    free_buf(tw);
    return rc;
  }
  return end_call(c, stream, RSB_OK);
}

static int gs_lap_common(int64_t ne, int nv, const int64_t* ev, const void* x, void* y, int f32,
                         int reps, double* ms, double* bytes, void* stream) {
  Ctx* pc = nullptr;
  int rc = begin_call(&pc, stream);
  if (rc) return rc;
  Ctx& c = *pc;
  int64_t V = 0;
  if ((rc = gs_setup(c, ne, nv, ev, &V))) return end_call(c, stream, rc);
  const size_t es = f32 ? 4 : 8;
  if ((rc = devbuf_reserve(c.gs_w, es * (size_t)(V + 1)))) return end_call(c, stream, rc);
  DevBuf tx, ty;
  const void* xd = x;
  void* yd = y;
  if (reps > 0) {  // benchmark: operands of its own
    if ((rc = devbuf_reserve(tx, es * (size_t)ne)) || (rc = devbuf_reserve(ty, es * (size_t)ne)))
      return end_call(c, stream, rc);
    RSB_CK(cudaMemsetAsync(tx.p, 0, es * (size_t)ne, c.s));
    xd = tx.p;
    yd = ty.p;
  } else {
    if (!is_device_ptr(x)) {
      if ((rc = devbuf_reserve(tx, es * (size_t)ne))) return end_call(c, stream, rc);
      RSB_CK(cudaMemcpyAsync(tx.p, x, es * (size_t)ne, cudaMemcpyHostToDevice, c.s));
      xd = tx.p;
    }
    if (!is_device_ptr(y)) {
      if ((rc = devbuf_reserve(ty, es * (size_t)ne))) return end_call(c, stream, rc);
      yd = ty.p;
    }
  }
  auto apply = [&]() {
    return gs_apply(f32, ne, nv, V, dptr<int32_t>(c.gs_ev32), dptr<int64_t>(c.gs_bptr),
                    dptr<int32_t>(c.gs_bucket), xd, c.gs_w.p, yd, c.s);
  };
  if (reps <= 0) {
    rc = apply();
    if (!rc && yd != y)
      if (cudaMemcpyAsync(y, yd, es * (size_t)ne, cudaMemcpyDeviceToHost, c.s))
        rc = rsb_set_error(RSB_ECUDA, "copy y");
  } else {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int w = 0; w < 3 && !rc; ++w) rc = apply();
    cudaEventRecord(e0, c.s);
    for (int i = 0; i < reps && !rc; ++i) rc = apply();
    cudaEventRecord(e1, c.s);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms) *ms = (double)t / reps;
    // vertex sums: bucket offsets, bucket entries, x once, w written; element
    // pass: vertex ids, bucket offsets, w and x read once, y written
    if (bytes)
      *bytes = 16.0 * (double)(V + 1) + 8.0 * (double)ne * nv + 3.0 * es * (double)ne +
               2.0 * es * (double)V;
  }
  rc = end_call(c, stream, rc);
  free_buf(tx);
  free_buf(ty);
  return rc;
}

extern "C" int rsb_laplacian_apply_gs(int64_t ne, int nv, const int64_t* ev, const double* x,
                                      double* y, void* stream) {
  if (!x || !y) return rsb_set_error(RSB_EINVAL, "x and y are needed");
  return gs_lap_common(ne, nv, ev, x, y, 0, 0, nullptr, nullptr, stream);
}

extern "C" int rsb_laplacian_apply_gs_f32(int64_t ne, int nv, const int64_t* ev, const float* x,
                                          float* y, void* stream) {
  if (!x || !y) return rsb_set_error(RSB_EINVAL, "x and y are needed");
  return gs_lap_common(ne, nv, ev, x, y, 1, 0, nullptr, nullptr, stream);
}

extern "C" int rsb_laplacian_bench_gs(int64_t ne, int nv, const int64_t* ev, int f32, int reps,
                                      double* ms_per_apply, double* useful_bytes, void* stream) {
  if (reps < 1) return rsb_set_error(RSB_EINVAL, "reps");
  return gs_lap_common(ne, nv, ev, nullptr, nullptr, f32 ? 1 : 0, reps, ms_per_apply,
                       useful_bytes, stream);
}

extern "C" const char* rsb_strerror(int code) {
  switch (code) {
    case RSB_OK: return "success";
    case RSB_EINVAL: return "invalid argument";
    case RSB_ENOMEM: return "device memory allocation failed";
    case RSB_ECUDA: return "CUDA error";
    case RSB_ENOCONV: return "a Fiedler solve stopped at its iteration cap";
    case RSB_ETIMEOUT: return "a bounded device wait gave up";
    case RSB_EDISCONNECTED: return "graph is disconnected";
    default: return "unknown error code";
  }
}

extern "C" const char* rsb_last_error_detail(void) { return g_detail.c_str(); }

extern "C" void rsb_release(void) {
  amg_release();
  for (int d = 0; d < 64; ++d) {
    Ctx* c = g_ctx[d];
    if (!c) continue;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(d);
    DevBuf* all[] = {&c->slice_ptr[0], &c->slice_ptr[1], &c->ent[0], &c->ent[1], &c->deg[0],
                     &c->deg[1], &c->gid[0], &c->gid[1], &c->home[0], &c->home[1],
                     &c->row_seg[0], &c->row_seg[1], &c->len, &c->slice_sz, &c->scan_tmp,
                     &c->tmp64, &c->newpos, &c->parent, &c->cmin, &c->ckey, &c->side, &c->units,
                     &c->tiles, &c->sunits, &c->stiles, &c->hist, &c->partials, &c->mom, &c->sbuf,
                     &c->cand[0], &c->cand[1], &c->cand[2], &c->seg_row0, &c->seg_nleft,
                     &c->seg_child0, &c->seg_p0, &c->seg_split, &c->seg_keystar, &c->seg_unit,
                     &c->seg_ncomp, &c->counters, &c->part_concat, &c->blk, &c->coords_cat,
                     &c->perm, &c->iperm, &c->rcb_home, &c->gs_count, &c->gs_cursor,
                     &c->gs_bptr, &c->gs_bucket, &c->gs_ev32, &c->gs_len, &c->gs_rowptr,
                     &c->gs_w, &c->gs_misc};
    for (DevBuf* b : all) free_buf(*b);
    for (int k = 0; k < 2; ++k) {
      PrecBufs& p = c->pb[k];
      DevBuf* pv[] = {&p.Q, &p.W0, &p.W1, &p.Y, &p.X, &p.R, &p.P, &p.AP, &p.Z0, &p.Z1};
      for (DevBuf* b : pv) free_buf(*b);
    }
    stage_clear(*c);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
    g_ctx[d] = nullptr;
    cudaSetDevice(cur);
  }
}

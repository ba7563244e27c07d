// noalloc.cu — rsb_laplacian_apply_noalloc: the Laplacian action y = L x of
// rsb_laplacian_apply for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code running while a framework's
// caching allocator has reserved the whole device (a raw allocation would fail
// or fragment that pool), code inside an allocation-sensitive region where the
// implicit device synchronisation of cudaMalloc/cudaFree is not allowed, or
// embedders that account for every device byte up front.  This entry point
// takes all of its scratch (the sliced-ELL copy of the graph and the scan
// workspace) from one statically sized device array that the library image
// carries, so it allocates nothing at call time.
//
// Costs and rules (also in include/rsb.h):
//   * the array is RSB_NOALLOC_SCRATCH_BYTES (32 MiB); every GPU on which the
//     library is loaded holds it until the process exits;
//   * graphs whose scratch would not fit are rejected with RSB_EINVAL;
//   * every call shares the one array and leaves its contents behind; what
//     must start at zero is cleared by each call; calls that overlap on the GPU
//     (different streams or threads) race on the array and must be ordered by
//     the caller;
//   * inputs and outputs must be device pointers (host pointers would need a
//     staging allocation) and the caller's stream is used directly;
//   * the call reads the entry count and the validation flag back to the host
//     and synchronises the caller's stream, so it cannot be issued inside a
//     stream capture at all;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it.
#include <string>

#include "rsb_internal.cuh"

#define RSB_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[RSB_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device (host-side name of the array
// is only a stand-in, never a device address).
static void* g_noalloc_addr[64] = {nullptr};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" int rsb_laplacian_apply_noalloc(const rsb_csr* g, const double* x, double* y,
                                           void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!g || !x || !y) return rsb_set_error(RSB_EINVAL, "NULL argument");
  if (g->n < 1 || g->n >= RSB_MAXN) return rsb_set_error(RSB_EINVAL, "n out of range");
  if (!on_device(g->row_ptr) || !on_device(x) || !on_device(y) ||
      (g->col && !on_device(g->col)) || (g->weight && !on_device(g->weight)) ||
      (g->gid && !on_device(g->gid)))
    return rsb_set_error(RSB_EINVAL, "rsb_laplacian_apply_noalloc takes device pointers only");
  int dev = 0;
  RSB_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return rsb_set_error(RSB_EINVAL, "device index");
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return rsb_set_cuda_error(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_addr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_noalloc_addr[dev];
  const int64_t n = g->n;
  const int64_t nsl = (n + 31) / 32;
  int64_t nnz = 0;
  RSB_CK(cudaMemcpyAsync(&nnz, g->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  if (nnz < 0 || (nnz > 0 && !g->col)) return rsb_set_error(RSB_EINVAL, "row_ptr / col");
  // scratch layout: flag | len | slice_sz | scan tmp | slice_ptr | ent (the
  // Laplacian action needs no per-row degree, gid or segment arrays)
  size_t off = 0;
  int* flag = (int*)(base + off);
  off += 256;
  int32_t* len = (int32_t*)(base + off);
  off += align256(sizeof(int32_t) * (size_t)n);
  int64_t* slice_sz = (int64_t*)(base + off);
  off += align256(sizeof(int64_t) * (size_t)(nsl + 1));
  const size_t scan_bytes = scan_tmp_bytes(nsl + 1);
  void* scan_tmp = base + off;
  off += align256(scan_bytes);
  int64_t* slice_ptr = (int64_t*)(base + off);
  off += align256(sizeof(int64_t) * (size_t)(nsl + 2));
  const size_t ent_off = off;
  // the entries need at least 4 B per stored entry; the exact padded count is
  // known after the slice scan and checked again below
  if (ent_off + 4 * (size_t)nnz > RSB_NOALLOC_SCRATCH_BYTES)
    return rsb_set_error(RSB_EINVAL, "graph too large for the 32 MiB no-allocation scratch");
  int rc;
  RSB_CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  if ((rc = launch_validate(g->row_ptr, g->col, g->weight, n, 0, flag, s))) return rc;
  if ((rc = launch_row_lengths(g->row_ptr, n, len, s))) return rc;
  if ((rc = launch_slice_widths(len, n, slice_sz, s))) return rc;
  RSB_CK(cudaMemsetAsync(slice_sz + nsl, 0, sizeof(int64_t), s));
  if ((rc = launch_scan_i64(slice_sz, slice_ptr, nsl + 1, scan_tmp, scan_bytes, s))) return rc;
  int64_t hv[2] = {0, 0};
  RSB_CK(cudaMemcpyAsync(&hv[0], slice_ptr + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaMemcpyAsync(&hv[1], flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  if ((int)hv[1] != 0) return rsb_set_error(RSB_EINVAL, "invalid graph");
  const int64_t total = hv[0];
  if (ent_off + 4 * (size_t)total > RSB_NOALLOC_SCRATCH_BYTES)
    return rsb_set_error(RSB_EINVAL, "graph too large for the 32 MiB no-allocation scratch");
  LevelGraph G;
  G.n = (int32_t)n;
  G.nslices = nsl;
  G.slice_ptr = slice_ptr;
  G.ent = (uint32_t*)(base + ent_off);
  G.deg = nullptr;
  G.gid = nullptr;
  G.home = nullptr;
  G.row_seg = nullptr;
  G.nent = total;
  if ((rc = launch_fill_sell(g->row_ptr, g->col, g->weight, g->gid, n, 0, 0, 0, G.slice_ptr,
                             G.ent, G.deg, G.gid, G.home, G.row_seg, s)))
    return rc;
  if ((rc = launch_spmv_f64(G, x, y, s))) return rc;
  RSB_CK(cudaStreamSynchronize(s));
  return RSB_OK;
}

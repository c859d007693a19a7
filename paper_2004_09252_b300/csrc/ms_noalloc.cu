// ms_crypt_pages_noalloc: the host-list page cipher with no allocation at
// call time.
//
// Who needs it: a caller on a page-fault path (the server thread that is
// resolving a client's fault and must hand back a decrypted page) cannot
// afford cudaMalloc there: it can implicitly synchronise the whole device,
// and it can fail outright when a caching allocator already holds the free
// device memory.  Such a caller creates its context beforehand (ms_init
// allocates) and then uses this entry point, which allocates nothing.
//
// The kernel is the same one-launch page kernel as ms_encrypt_pages.  Its
// scratch -- the device copy of the entry list and the status word the
// kernel reports bad entries in -- lives in one file-scope device array
// instead of the context's staging buffers.  That array is loaded with the
// library's device code and every GPU that loads the library keeps it until
// the process exits.
#include <cstring>
#include <mutex>

#include "ms_internal.h"

namespace {

constexpr size_t kScratchHeader = 256;  // bytes before the entry list; the status word is at 0
constexpr size_t kScratchBytes = kScratchHeader + (size_t)MS_NOALLOC_MAX_PAGES * sizeof(ms_page);

static __device__ __align__(256) unsigned char ms_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch[kMaxDevices] = {};  // device address of the array, per device

// Device address of the scratch array on `dev` (which must be current).  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up once per device and kept for the life of the process (a device
// reset, which unloads the array, is not supported afterwards).
int scratch_on(ms_ctx *c, int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return MS_ERANGE;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, ms_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return ms::cuda_fail(c, e == cudaSuccess ? cudaErrorUnknown : e);
    g_scratch[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch[dev];
  return MS_OK;
}

// Host-side entry checks without allocating: no NULL or misaligned address,
// and, when the context sets check_duplicates, no address listed twice.  The
// duplicate test uses one fixed open-addressing table (twice the largest list,
// so it never fills) whose slots count as empty unless they carry the current
// call's stamp; it is shared by all contexts under its own lock.
constexpr size_t kSeenSlots = 2 * (size_t)MS_NOALLOC_MAX_PAGES;
static_assert((kSeenSlots & (kSeenSlots - 1)) == 0, "table size must be a power of two");
struct SeenSlot {
  uint64_t addr;
  uint64_t stamp;
};
std::mutex g_seen_mu;
SeenSlot g_seen[kSeenSlots];
uint64_t g_seen_stamp = 0;

int check_entries(const ms_ctx *c, const ms_page *pages, size_t n) {
  if (!pages) return MS_EINVAL;
  for (size_t i = 0; i < n; ++i)
    if (pages[i].addr == 0 || (pages[i].addr & 15u)) return MS_EINVAL;
  if (!c->cfg.check_duplicates) return MS_OK;
  std::lock_guard<std::mutex> lk(g_seen_mu);
  const uint64_t stamp = ++g_seen_stamp;
  for (size_t i = 0; i < n; ++i) {
    const uint64_t a = pages[i].addr;
    size_t h = (size_t)((a >> 4) * 0x9E3779B97F4A7C15ull >> 40) & (kSeenSlots - 1);
    while (g_seen[h].stamp == stamp) {
      if (g_seen[h].addr == a) return MS_EINVAL;
      h = (h + 1) & (kSeenSlots - 1);
    }
    g_seen[h].addr = a;
    g_seen[h].stamp = stamp;
  }
  return MS_OK;
}

}  // namespace

extern "C" int ms_crypt_pages_noalloc(ms_ctx *c, int op, const ms_page *pages, size_t n) {
  using namespace ms;
  if (!c || !c->alive) return MS_ENOTINIT;
  if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
  if (n == 0) return MS_OK;
  if (n > MS_NOALLOC_MAX_PAGES) return MS_ERANGE;
  // The same checks as ms_encrypt_pages (addresses; repeated pages when the
  // context asks for it), made without allocating.
  int rc = check_entries(c, pages, n);
  if (rc != MS_OK) return rc;

  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  // The call waits for its own kernel and reads its status back; on a stream
  // that is being captured neither can happen, so refuse before touching it.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cap);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (cap != cudaStreamCaptureStatusNone) return MS_EINVAL;
  unsigned char *base = nullptr;
  rc = scratch_on(c, c->device, &base);
  if (rc != MS_OK) return rc;
  unsigned int *d_status = reinterpret_cast<unsigned int *>(base);
  ms_page *d_list = reinterpret_cast<ms_page *>(base + kScratchHeader);

  // The array keeps whatever the previous call left: the status word must
  // start at zero; the first n entries are overwritten below.
  e = cudaMemsetAsync(d_status, 0, sizeof(unsigned int), c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_list, pages, n * sizeof(ms_page), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  PageArgs a = make_args(c);
  a.pages = d_list;
  a.n_pages = n;
  a.status = d_status;
  e = launch_pages(c, a, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(c->sync_ev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  rc = wait_event(c, c->sync_ev, c->cfg.timeout_ms);
  if (rc != MS_OK) return rc;
  // A copy into pageable host memory returns only once it has completed; the
  // kernel is already done, so this waits for nothing but the 4-byte copy.
  unsigned int st = 0;
  e = cudaMemcpyAsync(&st, d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  return (st & kStatusBadEntry) ? MS_EINVAL : MS_OK;
}

/*
 * memshield.h -- C ABI of the B300 page cipher (MemShield, arXiv 2004.09252).
 *
 * What the library computes (MemShield Sec. 4.4, "GPU encryption"): every
 * operation acts on whole 4096-byte pages.  A page is XORed, in place, with
 * 64 ChaCha20 keystream blocks of 64 bytes.  Each block is derived from the
 * 256-bit master key and a 128-bit value made of the page's identity, the
 * client identity (PID) and the block's index 0..63 inside the page.
 * Encryption and decryption are the same operation.
 *
 * Field layout of the 128-bit value (the paper gives no order; this is the
 * library's fixed reading, in the RFC 8439 ChaCha20 state layout):
 *   word 12 = block index j (0..63), word 13 = low 32 bits of the page id,
 *   word 14 = high 32 bits of the page id, word 15 = the domain word (the
 *   paper's PID slot; ms_config.domain, 0 by default).
 * The round count is 20 (the paper's ChaCha20); 8 and 12 are accepted as
 * reduced-round variants.
 *
 * Memory: page addresses are device-accessible pointers (device memory, or
 * pinned host memory mapped into the device's address space), each 16-byte
 * aligned.  The caller owns page memory and must keep it valid and untouched
 * until ms_sync() returns for the submission.  A page must not appear twice in
 * one submission (two in-place updates of one page would race); re-encrypting
 * a page with the same (key, page id, domain) reuses its keystream, as in the
 * paper, which keeps no per-page version.
 *
 * Key: ms_init copies the key into device memory through a pinned bounce
 * buffer that it wipes before returning; afterwards the library holds the key
 * only on the device (the paper keeps it in the registers of a kernel that
 * never exits, Sec. 4.4; this library keeps it in a device buffer instead, so
 * launches can end).  Copies made by the CUDA driver itself are outside the
 * library's control.
 *
 * Errors: every int-returning call returns MS_OK (0) or a negative MS_E* code;
 * ms_strerror() names it.  n = 0 is a successful no-op.  Calls on one context
 * may come from several host threads; submissions are serialised internally.
 *
 * Contents:
 *   contexts            ms_init, ms_clone, ms_sync, ms_shutdown
 *   one launch          ms_encrypt_pages / ms_decrypt_pages (host list),
 *                       *_dev (device list), ms_crypt_pages_dom*, ms_crypt_range
 *   tickets             ms_submit_host, ms_poll, ms_wait
 *   host streaming      ms_crypt_host (copy engines), ms_crypt_host_inplace (in place over the link)
 *   shape and tuning    ms_get_shape / ms_set_shape, ms_autotune, ms_tune_save/load
 *   batched             ms_batch_* (persistent kernel, device queue, CUDA graphs)
 *   served              ms_server_* (continuous batching over a host working set)
 *   sliding window      ms_window_run, ms_window_run_resident, ms_window_run_ticketed
 *   resident workers    ms_resident_* (always-running kernels fed through mapped rings)
 *   allocation-free     ms_crypt_pages_noalloc
 *   fed                 ms_feed_* (one persistent kernel fed while it runs)
 *   measurement         ms_probe_int_pipes
 *   testing             ms_debug_inject_fault (host-side failure injection)
 */
#ifndef MEMSHIELD_H
#define MEMSHIELD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_PAGE_BYTES 4096u
#define MS_BLOCK_BYTES 64u
#define MS_BLOCKS_PER_PAGE 64u
#define MS_KEY_BYTES 32u

enum ms_status {
  MS_OK = 0,
  MS_EINVAL = -1,     /* bad argument: NULL, misaligned page, bad op/rounds/size */
  MS_ENOTINIT = -2,   /* NULL or shut-down context */
  MS_ENOMEM = -3,     /* host or device allocation failed */
  MS_ECUDA = -4,      /* a CUDA runtime call failed (ms_last_cuda_error gives the code) */
  MS_ETIMEDOUT = -5,  /* a bounded wait ran out; the work may still complete later */
  MS_EBUSY = -6,      /* admission refused: queue or staging budget full */
  MS_ERANGE = -7,     /* size beyond a stated maximum */
  MS_ESTARVED = -8    /* a fed kernel waited wait_ms for entries that never came, and left */
};

enum ms_op { MS_ENCRYPT = 0, MS_DECRYPT = 1 };

/* One page of a submission: where the bytes live and which id seeds its nonce. */
typedef struct ms_page {
  uint64_t addr;    /* device-accessible address of the 4096-byte page, 16-byte aligned */
  uint64_t page_id; /* nonce words 13..14 (the paper's page address) */
} ms_page;

/* A page with its own domain word (the paper's client PID, nonce word 15),
 * for callers that serve several clients through one context.  32 bytes. */
typedef struct ms_page_dom {
  uint64_t addr;     /* as in ms_page */
  uint64_t page_id;  /* as in ms_page */
  uint32_t domain;   /* nonce word 15 for this page (overrides ms_config.domain) */
  uint32_t reserved0;
  uint64_t reserved1;
} ms_page_dom;

typedef struct ms_ctx ms_ctx;

typedef struct ms_config {
  int device;                  /* CUDA device ordinal; -1 = the calling thread's current device */
  void *stream;                /* cudaStream_t to launch on (see use_stream) */
  uint32_t domain;             /* nonce word 15 (the paper's client PID); default 0 */
  uint32_t rounds;             /* 20 (default), or 8 / 12 */
  uint32_t list_capacity;      /* entries per host-list staging slot (default 65536) */
  uint32_t timeout_ms;         /* bound on every host-side wait (default 10000) */
  uint32_t blocks_per_thread;  /* 0 = default (4); else 1, 2 or 4 keystream blocks per thread */
  uint32_t threads_per_cta;    /* 0 = default (128); else 128, 256 or 512 */
  uint32_t dr_unroll;          /* 0 = default (rounds/2); else double rounds per loop trip: 1, 2 or rounds/2 */
  uint32_t check_duplicates;   /* nonzero: host-list calls reject a page address listed twice */
  uint32_t use_stream;         /* nonzero: launch on `stream` even when it is NULL (the legacy
                                  default stream); zero and stream == NULL: the library's own stream */
} ms_config;

/* Fill *cfg with the defaults listed above. */
void ms_config_default(ms_config *cfg);

/*
 * Create a context on cfg->device: copy the 32-byte master key to device
 * memory (key == NULL draws it from the OS CSPRNG, getrandom(2), as the paper
 * does, Sec. 4.4), create the stream and the staging buffers.  *out receives
 * the context; on failure *out is NULL and nothing is left allocated.
 */
int ms_init(ms_ctx **out, const uint8_t *key, const ms_config *cfg);

/*
 * A context with the same key as `ctx` (copied device to device: the key
 * never returns to host memory), the given domain (the nonce's PID word),
 * its own stream and staging, and ctx's launch shape and tuning.  For a
 * server with many clients: one clone per client PID, each with its own
 * stream.  Shut it down like any context.
 */
int ms_clone(ms_ctx *ctx, uint32_t domain, ms_ctx **out);

/*
 * Encrypt / decrypt (the same transform, Sec. 4.4) n pages listed in HOST
 * memory.  Every entry is checked first (addr != 0, addr % 16 == 0); one bad
 * entry fails the whole call with MS_EINVAL and launches nothing.  The list is
 * copied before the call returns (the caller may reuse it at once); the work
 * is queued on the context's stream and completes asynchronously: ms_sync()
 * waits for it.  Up to 1024 entries (512 with per-page domains) travel in the
 * kernel's parameters: one launch, no copy.  Longer lists, or any list on a
 * context whose shape the caller set, go through pinned staging slots of
 * list_capacity entries and one host-to-device copy per slot.
 */
int ms_encrypt_pages(ms_ctx *ctx, const ms_page *pages, size_t n);
int ms_decrypt_pages(ms_ctx *ctx, const ms_page *pages, size_t n);

/*
 * Same, with the entry list already in DEVICE memory (d_pages, 16-byte
 * aligned, owned by the caller, valid until ms_sync returns).  Entries are
 * checked on the device: a bad entry is skipped and the next ms_sync returns
 * MS_EINVAL; the good entries are still processed.
 */
int ms_encrypt_pages_dev(ms_ctx *ctx, const ms_page *d_pages, size_t n);
int ms_decrypt_pages_dev(ms_ctx *ctx, const ms_page *d_pages, size_t n);

/*
 * Per-page domain forms (Sec. 4.4: the seed includes the client's PID, so one
 * GPU serves several clients with distinct keystreams).  Host list (checked
 * and copied like ms_encrypt_pages) or device list (checked on the device).
 * Encryption and decryption are the same call.
 */
int ms_crypt_pages_dom(ms_ctx *ctx, const ms_page_dom *pages, size_t n);
int ms_crypt_pages_dom_dev(ms_ctx *ctx, const ms_page_dom *d_pages, size_t n);

/* The device address of pinned, mapped host memory (for page entries that the
 * kernels read and write in place); MS_EINVAL for any other pointer.  The
 * paper has no counterpart: its GPU module reaches the client's page through
 * a buffer shared with the server (Sec. 4.4). */
int ms_host_device_address(const void *host_ptr, uint64_t *dev_addr);

/*
 * Ticketed submission, Sec. 4.2-4.4: a faulting client stays stalled until
 * the server has its page decrypted, so completion is per request, not per
 * context.  The host list `pages` (checked and copied as for
 * ms_encrypt_pages; the page addresses may be device memory or pinned,
 * mapped host memory, which the kernel then reads and writes in place over
 * the host link) is queued as one launch on the context's stream, and
 * *ticket names it.  n = 0 gives a ticket that completes after everything
 * queued before it.  ms_poll: 1 done, 0 pending, < 0 error (MS_EINVAL for a
 * ticket never issued).  ms_wait: MS_OK, MS_ETIMEDOUT after timeout_ms, or an
 * error.  At most MS_TICKETS submissions may be pending: a submit whose ring
 * slot still belongs to a pending ticket returns MS_EBUSY (wait for older
 * tickets first).
 */
#define MS_TICKETS 4096
int ms_submit_host(ms_ctx *ctx, int op, const ms_page *pages, size_t n, uint64_t *ticket);
int ms_poll(ms_ctx *ctx, uint64_t ticket);
int ms_wait(ms_ctx *ctx, uint64_t ticket, uint32_t timeout_ms);

/*
 * Contiguous form: n_pages pages back to back at the device address d_base
 * (16-byte aligned); page k has id first_page_id + k.  No entry list is read.
 * MS_EINVAL when the ids would wrap past 2^64 - 1 (a wrapped id would reuse
 * another page's keystream).
 */
int ms_crypt_range(ms_ctx *ctx, int op, void *d_base, uint64_t first_page_id, size_t n_pages);

/*
 * Sec. 4.2 and 4.4: the server resolves a client's page fault only once the
 * GPU module has returned the decrypted page.  ms_sync waits, at most
 * cfg.timeout_ms, until all work submitted on this context has finished.
 * Returns MS_ETIMEDOUT if the bound ran out (the work is still queued; call
 * again), MS_EINVAL if a device-checked entry was bad since the last
 * ms_sync, MS_ESTARVED if a fed kernel gave up waiting, MS_ECUDA on a CUDA
 * error.  The context is held for the duration of the wait: other threads'
 * submissions on it wait too.  Threads that need completion of their own
 * requests without that use ms_submit_host and ms_wait.
 */
int ms_sync(ms_ctx *ctx);
/* ms_sync with its own bound instead of cfg.timeout_ms (0 = only check);
 * Sec. 4.2 and 4.4, as ms_sync. */
int ms_sync_for(ms_ctx *ctx, uint32_t timeout_ms);

/*
 * Sec. 4.4: the master key is kept only on the GPU (purged from the server's
 * memory), so nothing of it may remain once the module ends.  ms_shutdown
 * finishes outstanding work (bounded), overwrites the device key with zeros
 * and frees every resource.  ctx must not be used afterwards.  NULL is a
 * no-op.  MS_EBUSY (and nothing is freed) while a batch, feed, server or
 * resident worker set created on the context has not been destroyed.
 * MS_ETIMEDOUT (and nothing is touched: the context stays usable, call
 * again) when the queued work does not finish within timeout_ms.
 */
int ms_shutdown(ms_ctx *ctx);

/*
 * Launch shape of the page kernels (what the autotuner picks).  Not part of
 * the method: every shape computes the same bytes.
 *   blocks_per_thread  1, 2 or 4 keystream blocks per thread
 *   threads_per_cta    128, 256 or 512
 *   dr_unroll          double rounds per loop trip (1, 2, or all of them)
 *   rot_policy         0: rotations as funnel shifts; 1: rotations by 16 and 8
 *                      as byte permutes; 2..7: as 1, with some rotations by 12
 *                      and 7 done on the integer multiply pipe (x * 2^k, high
 *                      + low halves): 2 all of them, 3 the 7s, 4 the 12s,
 *                      5 the 7s of column rounds, 6 the 7s through one wide
 *                      multiply, 7 the 12s and 7s of column rounds
 *   hoist              1: the part of the first double round that does not
 *                      depend on the block counter (41 of 992 operations) is
 *                      computed once per page per thread and shared by its
 *                      blocks; needs blocks_per_thread >= 2, dr_unroll =
 *                      rounds / 2, rot_policy 0 or 1
 * ms_set_shape returns MS_EINVAL (and changes nothing) for a shape that is
 * not compiled for the context's round count.  Until a shape is set (here or
 * in ms_config), a one-launch call whose pages would not fill the GPU with
 * the default (or tuned: ms_autotune, ms_tune_load) shape runs with 1 block
 * per thread, which finishes small launches sooner, and host lists of up to
 * 1024 entries travel in the kernel parameters; a set shape is always used
 * as it is.
 */
typedef struct ms_shape {
  uint32_t blocks_per_thread;
  uint32_t threads_per_cta;
  uint32_t dr_unroll;
  uint32_t rot_policy;
  uint32_t hoist;
} ms_shape;

int ms_get_shape(const ms_ctx *ctx, ms_shape *out);
int ms_set_shape(ms_ctx *ctx, const ms_shape *shape);

/* Static English description of an ms_status code.  The paper has no
 * counterpart: it names no error conditions. */
const char *ms_strerror(int code);

/* The cudaError_t of the most recent MS_ECUDA on this context (0 if none). */
int ms_last_cuda_error(const ms_ctx *ctx);

/*
 * Host-side fault injection, for tests of error handling (no GPU fault is
 * ever caused).  Arms a one-shot failure: the (countdown + 1)-th call at a
 * site in site_mask behaves as if the CUDA runtime had returned cuda_error
 * there (the real call is skipped), so the entry point returns MS_ECUDA and
 * ms_last_cuda_error gives cuda_error.  site_mask 0 disarms.  Process-wide.
 */
enum ms_fault_site {
  MS_FAULT_LAUNCH = 1,  /* page-kernel launches (one-launch forms) */
  MS_FAULT_COPY = 2,    /* host->device copies of entry lists and host-streamed chunks */
  MS_FAULT_GRAPH = 4,   /* batched-form graph launches */
  MS_FAULT_SERVER = 8   /* a served wave's first copy: the server fails its pending requests */
};
int ms_debug_inject_fault(int site_mask, int countdown, int cuda_error);

/*
 * Host pages, streamed (end-to-end form).  n_pages pages back to back at the
 * HOST address host_base (pinned memory gives overlapped copies; pageable
 * memory works but serialises); page k has id first_page_id + k.  The range
 * is cut into chunks of chunk_bytes (a multiple of 4096, 0 = 16 MiB); chunk i
 * goes host->device, through the cipher and back on stream i % n_streams
 * (n_streams 1..4, 0 = 2) with its own device buffer, so copies in both
 * directions overlap the kernels.  Returns when the results are back in
 * host memory (bounded by timeout_ms per chunk).  MS_EINVAL when the ids
 * would wrap past 2^64 - 1.
 */
int ms_crypt_host(ms_ctx *ctx, int op, void *host_base, uint64_t first_page_id, size_t n_pages,
                  size_t chunk_bytes, int n_streams);

/*
 * Host pages, in place (Sec. 4.4's page transform applied where the page
 * lies; the paper instead copies each page into GPU memory and back).
 * n_pages (< 2^32) pages back to back at host_base, which must be pinned,
 * mapped host memory (cudaHostAlloc, or registered and mapped), 16-byte
 * aligned; page k has id first_page_id + k.  The kernel reads and writes the
 * pages over the host link with a bounded grid (16 CTAs of 512 threads, each
 * thread loading its next keystream block's bytes while it computes the
 * current one) -- no device buffer, no copy engine.  Asynchronous on the
 * context's stream like ms_crypt_range: the results are in host memory once
 * ms_sync returns.  MS_EINVAL for memory that is not pinned and mapped, a
 * misaligned base, or ids that would wrap past 2^64 - 1.
 */
int ms_crypt_host_inplace(ms_ctx *ctx, int op, void *host_base, uint64_t first_page_id, size_t n_pages);

/*
 * ---- Batched form (persistent kernel fed by a device work queue) ----
 *
 * Sec. 4.4: the GPU module's workers take pages from queues that many host
 * threads fill, so uneven lists of pages (from faults and evictions) share
 * the GPU.  Here requests are appended to a host queue buffer; a submit
 * copies it into a device work queue and launches one persistent grid
 * (sized to what fits on the GPU) whose CTAs claim `grab` pages at a time
 * with an atomic on the queue head until the queue is empty.  The launch is
 * a captured CUDA graph (head reset, then the kernel) unless use_graph is 0.
 * Two queue buffers alternate, so requests for the next batch can be added
 * while the previous one runs.
 *
 * Ownership: page memory stays the caller's and must stay valid until
 * ms_sync(ctx) returns after the submit; entries are copied by
 * ms_batch_add.  A page must not appear twice in one batch.  Destroy every
 * batch before ms_shutdown of its context.
 */
typedef struct ms_batch ms_batch;

#define MS_BATCH_MAX_CAPACITY (1u << 26)

typedef struct ms_batch_config {
  uint32_t capacity;     /* pages per batch (default 1 << 20, max MS_BATCH_MAX_CAPACITY) */
  uint32_t use_graph;    /* nonzero (default): launch through a captured CUDA graph */
  uint32_t grab;         /* pages a CTA claims per atomic; 0 = the context's tuned value */
  uint32_t ctas_per_sm;  /* persistent CTAs per SM; 0 = the tuned value (all that fit) */
  uint32_t per_page_domain; /* nonzero: queue entries carry a domain each (32 B, ms_batch_add_dom) */
} ms_batch_config;

typedef struct ms_batch_stats {
  uint64_t requests;       /* successful ms_batch_add calls */
  uint64_t pages;          /* pages added */
  uint64_t submits;        /* non-empty submits */
  uint64_t graph_launches; /* submits that launched the captured graph */
} ms_batch_stats;

void ms_batch_config_default(ms_batch_config *cfg);
/* Allocates two pinned + two device queue buffers of 256 + 16 * capacity bytes
 * (32 * capacity with per_page_domain) and, with use_graph, captures the CUDA
 * graph of each buffer, so that no submit pays for a capture (a later change
 * of the context's tuning recaptures at the next submit). */
int ms_batch_create(ms_ctx *ctx, const ms_batch_config *cfg, ms_batch **out);
/* Append one request (op is bookkeeping: encryption = decryption).  Entries are
 * checked on the host (MS_EINVAL).  MS_EBUSY: the batch is full, submit first;
 * MS_ERANGE: the request alone is larger than the batch capacity. */
int ms_batch_add(ms_batch *batch, int op, const ms_page *pages, size_t n);
/* Same with a domain (client PID) per page; the batch must have been created
 * with per_page_domain (else MS_EINVAL).  ms_batch_add on such a batch uses
 * the context's domain. */
int ms_batch_add_dom(ms_batch *batch, int op, const ms_page_dom *pages, size_t n);
/* Append n_requests requests at once: request r is op ops[r] on
 * pages[offsets[r] .. offsets[r + 1]) (offsets has n_requests + 1 entries).
 * Stops at the first request that fails (MS_EBUSY when the batch is full);
 * *added (may be NULL) receives the number of requests queued. */
int ms_batch_add_requests(ms_batch *batch, size_t n_requests, const int *ops, const uint64_t *offsets,
                          const ms_page *pages, size_t *added);
/* Copy the queued requests to the device and launch K2; asynchronous (ms_sync). */
int ms_batch_submit(ms_batch *batch);
int ms_batch_get_stats(const ms_batch *batch, ms_batch_stats *out);
/* Waits (bounded) for the batch's work, then frees it.  NULL is a no-op.
 * MS_ETIMEDOUT (nothing freed; call again) if the work does not finish. */
int ms_batch_destroy(ms_batch *batch);

/*
 * ---- Autotuner ----
 * Times every compiled K1 shape (blocks per thread, threads per CTA, unroll,
 * rotation policy) on sample_pages contiguous pages (0 = 65536, 256 MiB), then
 * K2's pages-per-claim (1..64) and CTAs per SM (all that fit, or half) on a
 * scattered list of the same pages, and makes the fastest the context's
 * shape.  It allocates (and frees) its own sample buffer; page contents do
 * not matter.  Takes seconds; call it once after ms_init.
 */
typedef struct ms_tune_result {
  ms_shape shape;        /* chosen K1 shape */
  double k1_gbs;         /* its throughput on the sample, page bytes per second / 1e9 */
  uint32_t grab;         /* chosen K2 pages per claim */
  uint32_t ctas_per_sm;  /* chosen K2 CTAs per SM */
  double queue_gbs;      /* K2 throughput on the scattered sample */
  uint32_t tried;        /* configurations timed */
} ms_tune_result;

int ms_autotune(ms_ctx *ctx, size_t sample_pages, ms_tune_result *out);
/* One-line text table: GPU name, SM count, rounds, K1 shape, K2 grab and CTAs/SM.
 * Load rejects (MS_EINVAL) a table made for another GPU or round count. */
int ms_tune_save(const ms_ctx *ctx, const char *path);
int ms_tune_load(ms_ctx *ctx, const char *path);

/*
 * ---- Served form (continuous batching over host pages) ----
 *
 * Stands in for the paper's server + data thread (Sec. 4.2-4.4): faults ask
 * for single pages to be decrypted, evictions hand over runs of pages to be
 * encrypted, and both are served from a working set in host RAM.  A server
 * thread admits requests in arrival order while the pinned staging budget
 * has room and none of the request's pages is already in flight (a request
 * touching an in-flight page waits for it, and so does any later request
 * sharing a page with a waiting one, so results do not depend on the mix;
 * requests on other pages go ahead).  Admitted requests form a wave:
 *   - worker threads copy its pages from the working set into pinned
 *     staging (the paper's data thread copying into the shared page);
 *   - the pages go host->device on one stream, through the page kernel and
 *     back device->host on a second stream, so the copies of consecutive
 *     waves overlap in both directions (double buffering, waves_in_flight);
 *   - when a wave's copy-back completes, its pages are copied into the
 *     working set, its staging is wiped if zero_staging is set (the paper
 *     zeroes the shared page after each transfer), and its requests
 *     complete.
 * A new wave is formed as soon as the pipeline has room, from whatever has
 * arrived: requests join while others are on the GPU (continuous batching).
 * mode = MS_SERVE_ONE_PER_LAUNCH makes every wave a single request (the
 * plain one-launch-per-request form, same machinery).
 *
 * The working set: n_pages pages of 4096 bytes at host_base (pinned memory
 * is not required but avoids extra copies); page index i uses page id i.
 * The caller must not touch a page while a request on it is pending.
 */
typedef struct ms_server ms_server;

/* MS_SERVE_CONTINUOUS over pinned, mapped memory with zero_copy_max_pages > 0
 * (the default): no wave is staged.  Short queues go through the in-place
 * lane (entries in the kernel parameters); longer ones form waves whose
 * entries take staging slots while their pages stay in place, as in
 * MS_SERVE_ZERO_COPY.  Over pageable memory, or with zero_copy_max_pages = 0,
 * every wave is staged as described above.  MS_SERVE_ONE_PER_LAUNCH always
 * stages.
 * MS_SERVE_ZERO_COPY: no staging copies; the kernel reads and writes the
 * working set directly over the host link (it must be pinned, mapped memory,
 * e.g. from cudaHostAlloc); the staging budget then only bounds the pages in
 * flight.  Requests are admitted the same way.
 * Every kernel that works on the working set in place runs on one stream of
 * the server, with a bounded grid (16 CTAs of 512 threads), the next
 * keystream block's bytes loaded while the current one is computed: on B300
 * that moves about 32 GB/s each way over the host link, where a grid of one
 * thread per block stays near 7.5 GB/s. */
enum ms_serve_mode { MS_SERVE_CONTINUOUS = 0, MS_SERVE_ONE_PER_LAUNCH = 1, MS_SERVE_ZERO_COPY = 2 };

typedef struct ms_server_config {
  uint64_t staging_bytes;    /* admission budget in pinned staging (default 256 MiB, multiple of 4096) */
  uint32_t max_wave_pages;   /* pages per wave at most (default staging pages / waves_in_flight) */
  uint32_t waves_in_flight;  /* pipeline depth, 1..8 (default 2) */
  uint32_t copy_threads;     /* gather/scatter worker threads, 0..32 (default 4) */
  uint32_t max_pending;      /* tickets not yet completed-and-reaped, at most (default 1 << 20) */
  uint32_t mode;             /* ms_serve_mode */
  uint32_t zero_staging;     /* nonzero: wipe staging pages after each wave */
  uint32_t max_request_pages;/* largest request accepted (default 4096; <= staging pages) */
  uint32_t idle_spin_us;     /* idle server thread polls this long before sleeping (default 20000:
                                a trickle of faults does not find it asleep) */
  uint32_t zero_copy_max_pages; /* continuous mode, working set in pinned mapped memory: the in-place
                                  lane.  While everything queued fits in this many pages (<= 512;
                                  also capped by max_wave_pages; 64 while a longer wave is in flight),
                                  the wave runs in place on the working set -- one launch with the
                                  entries in the kernel parameters, no entry copy -- and completes
                                  independently of the longer waves, which run in place too (see
                                  ms_serve_mode).  Default 512; 0 = lane off and every wave staged */
} ms_server_config;

typedef struct ms_server_stats {
  uint64_t requests_done;
  uint64_t pages_done;
  uint64_t waves;            /* kernel launches */
  uint64_t max_wave_requests;
  uint64_t max_wave_pages;
  uint64_t conflict_waits;   /* times the head request waited for an in-flight page */
  uint64_t budget_waits;     /* times the head request waited for staging room */
  uint64_t max_staged_pages; /* most staging slots ever in use (never above the budget) */
  uint64_t gather_ns;        /* server-thread time spent copying pages into staging */
  uint64_t scatter_ns;       /* ... and back into the working set */
  uint64_t inplace_waves;    /* waves run through the in-place lane (included in waves) */
  uint64_t staged_waves;     /* waves whose pages were copied through staging (included in waves) */
  uint64_t max_pass_ns;      /* longest single pass of the server thread's loop (completions,
                                admission, issue), its idle waits excluded; since the latest
                                ms_server_replay started (else since creation) */
  uint64_t replay_max_lag_ns;/* latest ms_server_replay: most a submission ran behind its schedule */
  uint64_t replay_late;      /* ... and how many submissions ran more than 1 ms behind */
} ms_server_stats;

void ms_server_config_default(ms_server_config *cfg);
/* Allocates the pinned staging, its device mirror and the entry lists, and
 * starts the server thread and the copy workers. */
int ms_server_create(ms_ctx *ctx, void *host_base, uint64_t n_pages, const ms_server_config *cfg,
                     ms_server **out);
/* Queue a request on pages page_index[0..n) of the working set (distinct
 * within the request, each < n_pages); *ticket identifies it.  MS_ERANGE: n
 * above max_request_pages; MS_EBUSY: max_pending tickets outstanding. */
int ms_server_submit(ms_server *srv, int op, const uint64_t *page_index, uint32_t n, uint64_t *ticket);
/* Same, for one client among several: its pages use `domain` as nonce word 15
 * (the paper's PID) instead of the context's domain. */
int ms_server_submit_dom(ms_server *srv, int op, uint32_t domain, const uint64_t *page_index, uint32_t n,
                         uint64_t *ticket);
/* 1 = done (its pages are back in the working set), 0 = pending, < 0 = error. */
int ms_server_poll(ms_server *srv, uint64_t ticket);
/* Wait up to timeout_ms for the ticket: MS_OK, MS_ETIMEDOUT or an error.
 * Polls with 1 us naps for about 50 us, then blocks; the calling thread's
 * timer slack is set to 1 us on its first nap so that the naps stay short. */
int ms_server_wait(ms_server *srv, uint64_t ticket, uint32_t timeout_ms);
/*
 * Open-loop replay, for measurement: request r (op ops[r], domain domains[r]
 * or the context's when domains is NULL, on page_index[offsets[r] ..
 * offsets[r + 1])) is submitted at arrival_s[r]
 * seconds after the start, however far behind the server is, and
 * latency_s[r] is its completion time minus that scheduled arrival (so
 * queueing delay counts: no coordinated omission).  *makespan_s receives the
 * time from the start to the last completion.  Waits at most timeout_ms
 * after the last arrival for completions.  Every request is checked before
 * the first is submitted (MS_EINVAL: empty request, bad op, page index out
 * of range or repeated within a request; MS_ERANGE: more than
 * max_request_pages).  On an error return after submission started,
 * requests still outstanding run to completion but no longer write to
 * latency_s, so the caller may free it at once.
 */
int ms_server_replay(ms_server *srv, size_t n_requests, const double *arrival_s, const int *ops,
                     const uint32_t *domains, const uint64_t *offsets, const uint64_t *page_index,
                     double *latency_s, double *makespan_s, uint32_t timeout_ms);
int ms_server_get_stats(const ms_server *srv, ms_server_stats *out);

/*
 * ---- Sliding-window clients (the fault / eviction stream of Sec. 4.3) ----
 *
 * Each client owns working-set pages [first_page, first_page + n_pages), all
 * ENCRYPTED (with the client's domain) when the run starts, and keeps a FIFO
 * window of pages in clear.  For every access in its trace (page numbers
 * relative to first_page):
 *   - in the window: a hit;
 *   - otherwise a fault: a one-page decrypt is submitted to the server and
 *     the client waits for it (the faulting process is stalled), then the
 *     page joins the window;
 *   - when the window holds more than window_pages pages, its oldest
 *     evict_batch pages are encrypted by one request the client does not
 *     wait for (evict_batch = 1 is the paper's policy; larger batches evict
 *     ahead of need).
 * Background eviction (the paper's conclusions, Sec. 7, propose encrypting
 * window pages in the background once the number of free slots drops below
 * a threshold): with background_free = T (1 .. window_pages - 1) each client
 * also runs an evictor thread.  Whenever fewer than T of the window's
 * window_pages slots are free, the evictor encrypts the oldest evict_batch
 * clear pages by one request, again until at least T slots are free, off the
 * faulting thread's path (a batch larger than the shortfall evicts ahead of
 * need); the overflow rule above stays as the fallback when the evictor runs
 * behind.  Client and evictor share the window under
 * one lock; a page's eviction is always submitted before any later fault on
 * it, and a faulting page joins the window only once it is decrypted.
 * Each client runs on its own thread; its requests use its domain (PID).
 * At the end every eviction has completed; the pages still in a client's
 * window are in clear and all its other pages are encrypted.
 */
typedef struct ms_window_config {
  uint32_t window_pages;     /* maximum pages in clear per client (Table 1: 4, 8, 16, 32) */
  uint32_t evict_batch;      /* pages encrypted per eviction request, 1..window_pages + 1 */
  uint32_t background_free;  /* 0: no background eviction; else T, 1..window_pages - 1 (above) */
  uint32_t sync_evict;       /* nonzero: the client waits for each of its own overflow evictions
                                before its next access, as the paper's per-client server thread
                                finishes an eviction before it takes the next fault; 0: evictions
                                are not waited for */
} ms_window_config;

typedef struct ms_window_client {
  uint32_t domain;         /* the client's PID: nonce word 15 of its pages */
  uint32_t reserved;
  uint64_t first_page;     /* its pages in the server's working set (ranges must not overlap) */
  uint64_t n_pages;
  const uint64_t *trace;   /* accessed page numbers, each < n_pages */
  uint64_t trace_len;
} ms_window_client;

typedef struct ms_window_stats {
  uint64_t accesses, hits, faults, evictions, evict_requests;  /* evictions: pages, both paths */
  uint64_t final_window_pages;
  double fault_p50_us, fault_p99_us, fault_max_us;  /* fault service time seen by the client */
  double elapsed_s;                                 /* the client's whole trace */
  uint64_t background_evictions;                    /* pages encrypted by the background evictor */
  uint64_t background_requests;                     /* its requests */
} ms_window_stats;

/* Run the clients to the end of their traces.  stats_out (may be NULL) gets one
 * entry per client; final_window_out (may be NULL) gets window_pages + 1 slots
 * per client with its final window, oldest first, padded with UINT64_MAX. */
int ms_window_run(ms_server *srv, const ms_window_config *cfg, const ms_window_client *clients, size_t n_clients,
                  ms_window_stats *stats_out, uint64_t *final_window_out, uint32_t timeout_ms);
/* Drain (bounded), stop the threads and free.  NULL is a no-op. */
int ms_server_destroy(ms_server *srv);

/*
 * ---- Resident workers (the paper's always-running GPU module, bounded) ----
 *
 * Sec. 4.4: the GPU module is a kernel that keeps running; each of its
 * workers (a CUDA block) takes pages from its own queue in host/device
 * mapped memory, filled by many host threads.  Here each worker is a
 * one-CTA kernel on its own stream polling its own ring in pinned, mapped
 * host memory; a request is one page (the fault path) whose bytes may live in
 * device memory or in pinned host memory (then the worker reads and writes
 * them over the host link: no copies, no launch per request).
 *
 * Bounds (no wait is unbounded): a worker leaves after idle_exit_us without
 * work, after max_run_ms in total, or at ms_resident_destroy; a submit or a
 * wait that finds it gone launches it again.  Requests are assigned to
 * workers round-robin; one worker serves its requests in order.  A page must
 * not be in flight twice.  ChaCha20 contexts only (cfg.rounds = 20).
 */
typedef struct ms_resident ms_resident;

typedef struct ms_resident_config {
  uint32_t workers;       /* worker CTAs, 1..64 (default 4) */
  uint32_t ring_entries;  /* requests per worker ring, a power of two, 4..2^20 (default 4096) */
  uint32_t idle_exit_us;  /* a worker leaves after this long without work (default 200000) */
  uint32_t max_run_ms;    /* and after this long in total, 1..600000 (default 10000) */
} ms_resident_config;

typedef struct ms_resident_stats {
  uint64_t requests;         /* submitted */
  uint64_t launches;         /* worker launches (first start and every restart) */
  uint64_t max_run_exits;    /* launches that ended by max_run_ms */
  uint64_t workers_running;  /* workers currently running */
  uint64_t replay_max_lag_ns;  /* last ms_resident_replay: the largest delay between a request's
                                  scheduled arrival and the submission of its last page */
} ms_resident_stats;

void ms_resident_config_default(ms_resident_config *cfg);
/* Allocates the rings (32 B per entry) and done words in pinned mapped memory. */
int ms_resident_create(ms_ctx *ctx, const ms_resident_config *cfg, ms_resident **out);
/* Queue one page; *ticket identifies it.  MS_EBUSY: the worker's ring is full. */
int ms_resident_submit(ms_resident *res, const ms_page_dom *page, uint64_t *ticket);
/* 1 = done (the page is written back), 0 = pending, < 0 = error. */
int ms_resident_poll(ms_resident *res, uint64_t ticket);
/* Polls with 0.5 us naps; the calling thread's timer slack is set to 1 us on
 * its first nap so that they stay short. */
int ms_resident_wait(ms_resident *res, uint64_t ticket, uint32_t timeout_ms);
int ms_resident_get_stats(const ms_resident *res, ms_resident_stats *out);
/* Stop the workers (bounded wait) and free.  NULL is a no-op. */
int ms_resident_destroy(ms_resident *res);
/*
 * Open-loop replay over a pinned, mapped host working set of n_pages pages at
 * host_base (page index i = page id i): request r (domain domains[r], or the
 * context's when NULL) on page_index[offsets[r] .. offsets[r + 1]) is
 * submitted at arrival_s[r], one resident request per page, and completes
 * when all its pages are done; a page still in flight from an earlier
 * request is waited for first.  latency_s[r] counts from the scheduled
 * arrival.  The working set is read and written in place over the host link.
 */
int ms_resident_replay(ms_resident *res, void *host_base, uint64_t n_pages, size_t n_requests,
                       const double *arrival_s, const uint32_t *domains, const uint64_t *offsets,
                       const uint64_t *page_index, double *latency_s, double *makespan_s, uint32_t timeout_ms);
/*
 * The sliding-window clients of ms_window_run, served by resident workers:
 * every fault is one resident request (decrypt, waited for) and every
 * eviction one request per page (encrypt, not waited for).  The working set
 * (n_pages pages at host_base, page index = page id) must be pinned, mapped
 * host memory; the workers read and write it in place.  A fault on a page
 * whose eviction is still running waits for that eviction first, so no page
 * is ever in flight twice.  Client ranges must lie inside the working set.
 */
int ms_window_run_resident(ms_resident *res, void *host_base, uint64_t n_pages, const ms_window_config *cfg,
                           const ms_window_client *clients, size_t n_clients, ms_window_stats *stats_out,
                           uint64_t *final_window_out, uint32_t timeout_ms);
/*
 * The same clients served by ticketed launches (ms_submit_host + ms_wait):
 * each client gets a clone of ctx (ms_clone) with its own domain and stream;
 * a fault is one launch waited for, an eviction one launch not waited for,
 * in place on the pinned, mapped working set.  A client's stream runs its
 * requests in submission order, so a fault on a page whose eviction is still
 * queued runs after it.
 */
int ms_window_run_ticketed(ms_ctx *ctx, void *host_base, uint64_t n_pages, const ms_window_config *cfg,
                           const ms_window_client *clients, size_t n_clients, ms_window_stats *stats_out,
                           uint64_t *final_window_out, uint32_t timeout_ms);

/*
 * Allocation-free variant of ms_encrypt_pages / ms_decrypt_pages.  The paper
 * has no counterpart: this is a library convenience.
 *
 * For callers that must not call cudaMalloc at the moment they encrypt or
 * decrypt -- typically code resolving a page fault, where an allocation can
 * stall the whole device or fail because a caching allocator holds the free
 * memory.  The context (created earlier by ms_init, which does allocate)
 * supplies the key, the stream and the launch shape; the call itself
 * allocates nothing, on the device or on the host.
 *
 * pages: host list of n entries, checked like ms_encrypt_pages: MS_EINVAL,
 * with nothing launched, on a NULL or misaligned address or, when the
 * context was created with check_duplicates, on an address listed twice.
 * n above MS_NOALLOC_MAX_PAGES returns MS_ERANGE and does nothing.
 *
 * Scratch: the entry list and the status word go to one file-scope device
 * array of 256 + 16 * MS_NOALLOC_MAX_PAGES bytes (256.25 KiB) that every GPU
 * using the library holds until the process exits.  The first call on a
 * device looks up that array's device address (set-up, once per device) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not use this entry point on a device after a
 * device reset (cudaDeviceReset).  All calls share the array: calls whose
 * work overlaps on the GPU (two contexts, two threads, two streams) race on
 * it and must be serialised by the caller.
 *
 * The call blocks: it waits (bounded by timeout_ms) for its kernel and reads
 * the kernel's status back.  It returns MS_OK, MS_EINVAL for a bad entry,
 * MS_ETIMEDOUT or MS_ECUDA; it returns MS_EINVAL without doing anything
 * while the context's stream is being captured.  After MS_ETIMEDOUT the
 * kernel may still be using the shared array: call ms_sync on the context
 * until it returns something other than MS_ETIMEDOUT before the next call to
 * ms_crypt_pages_noalloc on that device, from any context.
 */
#define MS_NOALLOC_MAX_PAGES 16384u
int ms_crypt_pages_noalloc(ms_ctx *ctx, int op, const ms_page *pages, size_t n);

/*
 * ---- Fed form: one persistent kernel drains a queue the host is still filling ----
 *
 * Sec. 4.4: the GPU module's workers consume queues that host threads keep
 * filling.  ms_feed_create allocates a device queue of `capacity` entries
 * and its pinned host copy.  ms_feed_open launches one persistent K2 grid on
 * the context's stream over the empty queue.  ms_feed_add_requests appends
 * requests (as ms_batch_add_requests) and, every `chunk` entries, publishes
 * them: a copy of the new entries, then a copy of the new count, on the
 * feed's own stream.  The kernel claims only published entries and works
 * through each claim as it is published.  ms_feed_close publishes the rest
 * and marks the feed closed; the kernel drains it and exits, and
 * ms_sync(ctx) waits for that.  A closed feed can be opened again.
 *
 * While open, the grid holds every SM.  Bounded: a CTA that waits wait_ms
 * for entries that are not published leaves and sets a status bit, and the
 * next ms_sync returns MS_ESTARVED.  A feed holds `capacity` entries in all
 * (MS_ERANGE beyond); open another for more.  Entries are checked on the
 * host (MS_EINVAL); pages must not repeat within a feed.  Destroy every feed
 * before ms_shutdown of its context.
 */
typedef struct ms_feed ms_feed;

typedef struct ms_feed_config {
  uint32_t capacity;  /* entries per feed (default 1 << 20, max MS_BATCH_MAX_CAPACITY) */
  uint32_t chunk;     /* entries per publication (default 16384, at least 1024) */
  uint32_t wait_ms;   /* longest wait of the kernel for a publication (default 2000, max 600000) */
  uint32_t grab;      /* largest claim per atomic; 0 = the context's tuned value */
} ms_feed_config;

typedef struct ms_feed_stats {
  uint64_t requests, pages, publications;
  uint64_t grid;      /* persistent CTAs of the last run */
  uint64_t runs, closes;
} ms_feed_stats;

void ms_feed_config_default(ms_feed_config *cfg);
/* Allocates 2 x 16 B x capacity (pinned + device) and loads the kernel, in
 * the context's current shape, so that a run pays for neither; launches
 * nothing. */
int ms_feed_create(ms_ctx *ctx, const ms_feed_config *cfg, ms_feed **out);
/* Launch the kernel over an empty queue, after the previous run (if any) has
 * drained (bounded wait).  MS_EBUSY if already open. */
int ms_feed_open(ms_feed *feed);
/* Request r is pages[offsets[r] .. offsets[r + 1]); stops at the first request
 * that fails; *added (may be NULL) receives the number appended.  MS_EINVAL
 * when the feed is not open.  A run holds `capacity` entries in all. */
int ms_feed_add_requests(ms_feed *feed, size_t n_requests, const int *ops, const uint64_t *offsets,
                         const ms_page *pages, size_t *added);
/* Publish what is left and close; idempotent. */
int ms_feed_close(ms_feed *feed);
int ms_feed_get_stats(const ms_feed *feed, ms_feed_stats *out);
/* Close if open, wait (bounded) for the kernel, free.  NULL is a no-op. */
int ms_feed_destroy(ms_feed *feed);

/*
 * ---- Measurement: integer pipe rates (the paper has no counterpart) ----
 *
 * Sustained rates of the 32-bit op classes the cipher is built from, alone
 * and in 1:1 mixes, on `device`: a grid of 4 CTAs of 256 threads per SM,
 * each thread 8 independent chains of 16384 operations, timed with CUDA
 * events over the whole GPU.  The rates bound the
 * page kernels (their roofline); bench.py reports them.  Fills out[0 ..
 * MS_PIPE_CLASSES - 1] in the order of the enum.  Allocates and frees its
 * own scratch; takes about a second.
 */
enum {
  MS_PIPE_ADD = 0,      /* add.u32 */
  MS_PIPE_XOR = 1,      /* xor.b32 (LOP3) */
  MS_PIPE_SHF = 2,      /* shf.l.wrap.b32 (funnel-shift rotate) */
  MS_PIPE_PRMT = 3,     /* prmt.b32 (byte permute) */
  MS_PIPE_MAD = 4,      /* mad.lo.u32 */
  MS_PIPE_MULHI = 5,    /* mul.hi.u32 */
  MS_PIPE_XOR_MAD = 6,  /* xor and mad.lo, 1:1 */
  MS_PIPE_SHF_MAD = 7,  /* shf and mad.lo, 1:1 */
  MS_PIPE_XOR_ADD = 8,  /* xor and add, 1:1 */
  MS_PIPE_XOR_SHF = 9,  /* xor and shf, 1:1 */
  MS_PIPE_CLASSES = 10
};

typedef struct ms_pipe_rate {
  int32_t op_class;         /* MS_PIPE_* */
  int32_t reserved;
  double lanes_per_sm_clk;  /* tops / (SMs x sm_mhz): lane operations per SM per clock */
  double sm_mhz;            /* SM clock seen during the run (clock64 vs globaltimer) */
  double tops;              /* whole-GPU lane operations per second / 1e12 (CUDA events) */
} ms_pipe_rate;

/* MS_EINVAL: bad device or out == NULL or n_out < MS_PIPE_CLASSES. */
int ms_probe_int_pipes(int device, ms_pipe_rate *out, size_t n_out);

#ifdef __cplusplus
}
#endif

#endif /* MEMSHIELD_H */

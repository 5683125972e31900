/*
 * elsar.h -- C ABI of libelsar, a B300 (sm_103a) GPU implementation of the
 * in-memory hot path of ELSAR, the learned partition-and-concatenate sort of
 * "Parallel External Sorting of ASCII Records Using Learned Models"
 * (arXiv 2305.05671).
 *
 * Records are fixed 100-byte ASCII records with a 10-byte key at offset 0
 * (the paper's benchmark format, Sec. 7.1).  The result of every sort is the
 * input records stably sorted by memcmp on the key (Sec. 7.1 methodology):
 * equal keys stay in input order.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers (CUDA global memory) owned by the
 *    caller; h_* are host pointers owned by the caller.  The library keeps no
 *    reference to any buffer after a call returns.
 *  - Record buffers must be 4-byte aligned; input and output must not
 *    overlap.  Workspace and model buffers must be 256-byte aligned.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) unless stated otherwise.  Some calls read a few bytes back
 *    to the host (stated per call) and therefore synchronise `stream`.
 *  - Errors are returned as an elsar_status; nothing is thrown and nothing
 *    aborts.  elsar_last_error() gives a message for the calling thread.
 *  - Supported: 0 <= n < 2^32 records.  Larger n returns ELSAR_EUNSUPPORTED.
 *  - The library allocates no device memory: scratch lives in the caller's
 *    workspace (size from elsar_workspace_size).  The one exception is
 *    elsar_sort_noalloc, whose scratch is a fixed array of
 *    ELSAR_NOALLOC_SCRATCH_BYTES (16 MiB) compiled into the library, held on
 *    every GPU that loads it until the process exits.
 */
#ifndef ELSAR_H
#define ELSAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ELSAR_RECORD_BYTES 100
#define ELSAR_KEY_BYTES 10

typedef struct CUstream_st* elsar_stream_t; /* same type as cudaStream_t */

typedef enum elsar_status {
  ELSAR_OK = 0,
  ELSAR_EINVAL = 1,       /* bad argument (null/misaligned pointer, bad parameter) */
  ELSAR_ENOMEM = 2,       /* a caller buffer (workspace, model) is too small */
  ELSAR_ECUDA = 3,        /* a CUDA call failed; elsar_last_error() has the CUDA message */
  ELSAR_ETIMEOUT = 4,     /* a device-side bounded wait gave up (reported in the status word) */
  ELSAR_EUNSUPPORTED = 5, /* n >= 2^32 or another unsupported size */
  ELSAR_EMODEL = 6        /* the model buffer does not hold a fitted model */
} elsar_status;

typedef enum elsar_model_kind {
  ELSAR_MODEL_RMI = 0,  /* the paper's RMI of linear models (Sec. 3.1) */
  ELSAR_MODEL_MLP = 1,  /* monotone MLP CDF trained on the GPU; the RMI is its fallback */
  ELSAR_MODEL_RADIX = 2 /* no model: equal-width slices of the printable key domain, the
                           radix-based partitioning the paper compares with (Sec. 3, Sec. 3.3) */
} elsar_model_kind;

/* Checks that decide whether a requested network is used (model_kind MLP);
 * skip_checks is an OR of the ones to leave out (0 = all three apply). */
typedef enum elsar_check {
  ELSAR_SKIP_BOUNDARY = 1, /* F of the smallest / largest sample key within 1/16 of 0 / 1 */
  ELSAR_SKIP_JUDGE = 2,    /* held-out sample at least as balanced as under the RMI */
  ELSAR_SKIP_IMBALANCE = 4 /* full-data largest partition at most 1.1 x the mean */
} elsar_check;

typedef enum elsar_balance {
  ELSAR_BALANCE_PAPER = 0,  /* partition p = min(P-1, floor(P * F(x)))  (Algorithm 1 reader loop) */
  ELSAR_BALANCE_REFINED = 1 /* cuts at the fine-bin boundaries closest to p*N/P (exact counts) */
} elsar_balance;

typedef enum elsar_schedule {
  ELSAR_SCHED_PER_PARTITION = 0, /* one sort launch per partition */
  ELSAR_SCHED_PERSISTENT = 1     /* one persistent kernel over a work queue of all partitions */
} elsar_schedule;

/* Parameters.  Zero fields take the defaults noted; elsar_default_params
 * fills them explicitly. */
typedef struct elsar_params {
  uint32_t num_partitions; /* P, power of two in [1, 65536]; default 1024 */
  uint32_t fine_bins_log2; /* log2 B of the model's fine bins; 0 = about 1024 records per bin,
                              clamped to [max(log2 P, 6), 20]; must be >= log2 P, <= 22 */
  uint32_t leaf_target;    /* T: an RMI node splits when it holds more than 2T sample keys; 0 = 16 */
  uint32_t max_depth;      /* RMI depth cap; 0 = 32 */
  uint32_t model_kind;     /* elsar_model_kind; default RMI */
  uint32_t balance;        /* elsar_balance; default REFINED */
  uint32_t schedule;       /* elsar_schedule; default PERSISTENT */
  uint32_t tile_pairs;     /* max pairs one CTA sorts in shared memory; 0 = tuned default */
  uint64_t sample_size;    /* S; 0 = 1% of n within [1000, 10^7] (Sec. 3.1, Sec. 6); must be < 2^24 */
  uint64_t seed;           /* seed of the key sample (SplitMix64 counter stream) */
  uint32_t skip_checks;    /* OR of elsar_check values: network checks to leave out; default 0 */
  uint32_t key_bytes;      /* l in [1, 10]: the key is the first l bytes of each record; 0 = 10.  Keys
                              shorter than the longest (variable-length keys, Sec. 4) are padded with
                              0 bytes, which sort below every printable character; the bytes after the
                              first l are payload and are not compared. */
  uint64_t wait_limit_cycles; /* limit of every device-side bounded wait of the bulk-copy pipelines
                                 (classify, scatter), in SM clock cycles; 0 = 2e9 (about a second).
                                 A wait that runs out makes the call return ELSAR_ETIMEOUT. */
} elsar_params;

/* Per-call measurements, filled when a non-NULL pointer is passed.  Passing
 * one makes the call record CUDA events and synchronise `stream` at the end. */
typedef struct elsar_stats {
  float pass_ms[8];     /* 0 fit, 1 classify+histogram, 2 scan/cuts/items, 3 scatter, 4 sort+gather */
  uint32_t launches;    /* kernels launched by the call */
  uint32_t num_items;   /* work items of the sort pass */
  uint32_t oversize_items;
  uint32_t model_nodes; /* RMI nodes */
  uint64_t max_partition;
  uint64_t max_bin;
  uint32_t model_used;      /* elsar_model_kind that classified the records */
  uint32_t fallback_reason; /* MLP asked for but not used: 1 boundary check (F of the smallest / largest
                               sample key not within 1/16 of 0 / 1), 2 less balanced than the RMI on a
                               held-out sample, 3 full-data partition imbalance above 1.1; 0 otherwise */
  /* the network's checks (model_kind MLP; zero otherwise): the judge's J buckets, the held-out keys
     in the largest bucket under the RMI and under the network, F at the first and last knot */
  uint32_t judge_buckets, judge_rmi_max, judge_mlp_max, reserved;
  float F_first_knot, F_last_knot;
} elsar_stats;

/* Fill *p with the defaults. */
void elsar_default_params(elsar_params* p);

/* Bytes of workspace elsar_sort needs for n records with these parameters
 * (elsar_fit_model, elsar_partition and elsar_sort_partitions need no more). */
size_t elsar_workspace_size(uint64_t n, const elsar_params* p);

/* Bytes of the device model buffer (fitted CDF model + fine-bin splitters). */
size_t elsar_model_size(uint64_t n, const elsar_params* p);

/*
 * Train the CDF model (Sec. 3.1) on a uniform key sample of d_records:
 * S sample positions mulhi64(SplitMix64_k(seed), n), their keys encoded in
 * base 95 (Sec. 4), sorted, an RMI of linear models fitted on the sorted
 * sample, then the B-1 fine-bin splitters of the model (the smallest key
 * encoding whose fine bin floor(B*F) is at least q).  Writes d_model
 * (elsar_model_size bytes).  Asynchronous for the RMI and RADIX kinds (the
 * RMI's levels run in a device-side loop: a graph whose while-node repeats
 * them until a level has no children); the network reads its judge counts
 * back, so model_kind MLP synchronises `stream`.
 * Errors: EINVAL (null/misaligned pointers, bad params, n == 0), ENOMEM
 * (buffers too small), EUNSUPPORTED (n >= 2^32), ECUDA.
 */
elsar_status elsar_fit_model(const void* d_records, uint64_t n, const elsar_params* p, void* d_model,
                             size_t model_bytes, void* d_ws, size_t ws_bytes, elsar_stream_t stream);

/*
 * Model-based partitioning (Sec. 3.3, Algorithm 1 reader loop, Eq. 1): for
 * every record, the key is packed into a 16-byte pair {hi = big-endian key
 * bytes 0-7; lo = (big-endian key bytes 8-9) << 32 | record index} and
 * classified by the model into a fine bin q; bins are counted, scanned, the
 * partitions cut (paper rule or refined rule) and the pairs scattered so that
 * d_pairs holds them grouped by fine bin in bin order (hence by partition, and
 * by model sub-bucket within each partition).
 * Outputs: d_pairs (n * 16 bytes, 16-byte aligned), d_bin_offsets (B+1 u32:
 * start of each fine bin in d_pairs), d_part_offsets (P+1 u64: start of each
 * partition, Sec. 3.5 write offsets).  Order inside one bin is unspecified.
 * Errors: EINVAL, ENOMEM, EMODEL (d_model not fitted for these params), ECUDA.
 */
elsar_status elsar_partition(const void* d_model, const void* d_records, uint64_t n, const elsar_params* p,
                             void* d_pairs, uint32_t* d_bin_offsets, uint64_t* d_part_offsets, void* d_ws,
                             size_t ws_bytes, elsar_stream_t stream);

/*
 * Sort every partition and concatenate (Sec. 3.4, Sec. 3.5): each fine bin of
 * d_pairs (as laid out by elsar_partition) is sorted in shared memory by
 * (key, record index), and the 100-byte records are gathered in that order
 * into d_out (n * 100 bytes).  d_pairs is overwritten with the sorted pairs
 * when a bin needs the multi-pass path; otherwise it is left as is.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
elsar_status elsar_sort_partitions(const void* d_records, uint64_t n, const elsar_params* p, void* d_pairs,
                                   const uint32_t* d_bin_offsets, void* d_out, void* d_ws, size_t ws_bytes,
                                   elsar_stream_t stream);

/*
 * The whole method on one record set resident in device memory:
 * elsar_fit_model, elsar_partition and elsar_sort_partitions back to back,
 * with their buffers carved from d_ws.  d_out receives the sorted records.
 * With stats == NULL and model_kind RMI or RADIX the call is asynchronous:
 * it enqueues the work on `stream` and returns; a device-side wait that gave
 * up (ELSAR_ETIMEOUT) is then kept in the workspace and reported by
 * elsar_wait.  With stats, or with model_kind MLP (its checks read counts
 * back), it synchronises `stream` and reports ELSAR_ETIMEOUT itself.
 * Without stats (RMI or RADIX) the call can be captured into a caller's CUDA
 * graph, after one call outside any capture (that call sets the kernels'
 * shared-memory limits); inside a capture the RMI's levels are launched as a
 * fixed sequence (empty levels exit at once) instead of the device loop.
 * Errors: as the three calls.
 */
elsar_status elsar_sort(const void* d_in, void* d_out, uint64_t n, const elsar_params* p, void* d_ws,
                        size_t ws_bytes, elsar_stream_t stream, elsar_stats* stats);

/*
 * End-to-end convenience: host records in, host records out.  Copies
 * h_in to d_in, sorts into d_out, copies d_out to h_out, all on `stream`
 * (pinned host buffers make the copies asynchronous DMA).  Synchronises
 * and reports like elsar_wait.
 */
elsar_status elsar_sort_host(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_in,
                             void* d_out, void* d_ws, size_t ws_bytes, elsar_stream_t stream);

/*
 * elsar_sort_host without waiting: the copy in, the sort (asynchronous, as
 * elsar_sort without stats; model_kind MLP waits for its checks) and the
 * copy out are enqueued on `stream` and the call returns.  With pinned host
 * buffers the copies are DMA transfers, so sets sorted on different streams
 * overlap one set's copy out with another's copy in (the host link carries
 * both directions at once).  The host and device buffers must stay valid
 * until the stream reaches the end of the call; elsar_wait(d_ws) then waits
 * for it and reports a device-side timeout.  No paper counterpart.
 * Errors: EINVAL (null host buffers), and as elsar_sort.
 */
elsar_status elsar_sort_host_async(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_in,
                                   void* d_out, void* d_ws, size_t ws_bytes, elsar_stream_t stream);

/*
 * Status of the asynchronous calls on workspace d_ws (ws_bytes >= 140, the
 * control words that open every workspace): synchronises `stream`, then
 * returns ELSAR_ETIMEOUT if a device-side bounded wait gave up in any
 * elsar_sort call on this workspace since the last check (that call's output
 * is not valid; later calls are unaffected: each clears its own status at
 * its start), and clears the report; ELSAR_OK otherwise.  A workspace no call
 * has used yet reports ELSAR_OK.  Errors: EINVAL (null, not 256-byte aligned
 * or too small), ECUDA.
 */
elsar_status elsar_wait(void* d_ws, size_t ws_bytes, elsar_stream_t stream);

/*
 * Out of core: n records in pinned host memory (h_in, allocated with
 * cudaHostAlloc / cudaMallocHost or registered with cudaHostRegister, so the
 * GPU can read it) sorted into h_out (pinned as well, not overlapping h_in)
 * with no more device memory than the workspace d_ws (ws_bytes is the device
 * budget).  The paper's external sort (Algorithm 1, Sec. 3.2-3.5) with host
 * memory in the place of its files:
 *   fit     the CDF model (model_kind; the network falls back to the RMI as in
 *           elsar_sort) from a sample read from host memory;
 *   pass 1  chunks copied in, classified, counted: the exact fine-bin
 *           histogram gives the partition cuts and the write offsets (Sec. 3.5);
 *   pass 2  chunks copied in again, split stably by partition on the GPU and
 *           copied out into their partitions' ranges of h_out, appended in
 *           input order (the fragment files of Sec. 3.3);
 *   sort    runs of consecutive partitions that fit the budget are copied in,
 *           sorted (each run with its own model, as LearnedSort does per
 *           partition, Sec. 3.4) and copied back in place.
 * Copies run on side streams overlapped with the kernels.  Synchronises.
 * Needs ws_bytes >= elsar_ooc_min_workspace(n, p).  A partition larger than
 * what the budget can sort at once returns ELSAR_EUNSUPPORTED (use more
 * partitions).  Errors: EINVAL (not pinned host memory, overlap), ENOMEM, ECUDA.
 */
typedef struct elsar_ooc_stats {
  float phase_ms[4];   /* 0 fit, 1 pass 1 (histogram), 2 pass 2 (split), 3 partition sorts */
  uint64_t h2d_bytes, d2h_bytes;
  uint32_t chunks, groups;
  uint64_t chunk_records, group_records;
  uint32_t model_used, fallback_reason;
  uint64_t max_partition;
} elsar_ooc_stats;

size_t elsar_ooc_min_workspace(uint64_t n, const elsar_params* p);
elsar_status elsar_sort_ooc(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_ws,
                            size_t ws_bytes, elsar_stream_t stream, elsar_ooc_stats* stats);

/*
 * Many independent record sets in one CUDA-graph-captured launch sequence
 * (the batched form of the method; the paper sorts one file at a time and
 * balances uneven partitions with dynamic thread scheduling, Sec. 7.3 -- here
 * all sets' work items feed one persistent kernel).  Every set is sorted on
 * its own, with its own model: a 1 % sample (seed + k for set k), its own RMI
 * (Sec. 3.1) and its own fine bins; all sets share the passes.  Set k's
 * sorted records go to d_out[k].
 *
 * elsar_batch_create builds a plan for fixed buffers and sizes: it uploads
 * per-set tables into the workspace, and captures the whole sequence into a
 * CUDA graph.  With tile_pairs == 0 it first autotunes -- the tile size, then
 * the fine-bin density of each size class of sets (fewer than 2^15 records,
 * fewer than 2^18, larger) -- by timing candidate graphs on the caller's
 * data; the choice is cached per device and workload shape for the process
 * (and in the file named by the environment variable ELSAR_TUNE_CACHE, if
 * set).  Creation synchronises.  elsar_batch_run launches the graph on
 * `stream` (asynchronous); elsar_batch_wait synchronises `stream` and reports
 * a device-side timeout.  The plan keeps the buffer pointers: they must stay
 * valid, and run/wait calls on one plan must not overlap.
 * Limits: 1 <= num_sets <= 2^24, every n[k] > 0, the sum of n[k] < 2^32.
 * Errors: EINVAL, ENOMEM (workspace below elsar_batch_workspace_size),
 * EUNSUPPORTED, ECUDA.
 */
typedef struct elsar_batch elsar_batch;

typedef struct elsar_batch_info {
  uint32_t tile_pairs;              /* pairs per shared-memory tile chosen */
  uint32_t records_per_bin_log2[3]; /* fine-bin density chosen per size class */
  uint64_t total_records, total_bins, sample_keys;
  uint32_t launches;    /* kernels in the captured sequence */
  uint32_t tuning_runs; /* candidate graphs timed by the autotuner (0 if cached or fixed) */
  float tuning_ms[16];  /* their times */
} elsar_batch_info;

size_t elsar_batch_workspace_size(const uint64_t* n, uint32_t num_sets, const elsar_params* p);
elsar_status elsar_batch_create(const void* const* d_in, void* const* d_out, const uint64_t* n, uint32_t num_sets,
                                const elsar_params* p, void* d_ws, size_t ws_bytes, elsar_stream_t stream,
                                elsar_batch** out);
elsar_status elsar_batch_run(elsar_batch* b, elsar_stream_t stream);
elsar_status elsar_batch_wait(elsar_batch* b, elsar_stream_t stream);
elsar_status elsar_batch_describe(const elsar_batch* b, elsar_batch_info* info);
void elsar_batch_destroy(elsar_batch* b);

/*
 * The learned CDF network (model_kind = ELSAR_MODEL_MLP) on its own, for
 * inspection and parity checks.  It is not in the paper, whose model
 * (Sec. 3.1) is the RMI; its definition: 12 features of a key encoding x are
 * ramps between 13 sorted-sample knots T (phi_m = clamp(x - T_m, 0, W_m) / W_m
 * with W_m = T_{m+1} - T_m, formed exactly then scaled in FP64 and rounded to
 * FP32), two hidden layers of 32 with sigma(z) = 0.5 + 0.5 z / (1 + |z|), an
 * output z = b3 + sum_j w3_j h2_j + sum_m v_m phi_m (a linear skip from the
 * features), F = clamp(z, 0, 1); all weights (W1, W2, w3, v) are
 * non-negative, so F is monotone.  Parameters are 1517 floats laid out
 * W1[32][12], b1[32], W2[32][32], b2[32], w3[32], b3, v[12].  Training starts
 * from F = sum(phi) / 12 (the interpolation of the sample CDF between the
 * knots) and takes 400 Adam steps on minibatches of 8192 sample keys, the
 * learning rate decayed from 1e-3 to 1e-5 by a half cosine.
 *
 * elsar_mlp_eval: F of each key encoding, FP32 (d_w 1517 floats, d_knots 13
 *   u64, d_x n u64 encodings, d_F n floats).  Asynchronous.
 * elsar_mlp_grad: gradient of mean((F - y)^2) over n samples, FP32 with a
 *   fixed summation order (d_y n floats, d_grad 1517 floats); needs
 *   elsar_mlp_grad_workspace(n) bytes of scratch.  Asynchronous.
 * elsar_mlp_splitters: the 2^log2B fine-bin splitters of the network
 *   (t[0] = 0; t[q] = smallest encoding whose bin floor(2^log2B F) >= q, then
 *   made non-decreasing).  Asynchronous.
 * Errors: EINVAL for null pointers or n >= 2^32; ECUDA.
 */
size_t elsar_mlp_grad_workspace(uint64_t n);
elsar_status elsar_mlp_eval(const float* d_w, const uint64_t* d_knots, const uint64_t* d_x, uint64_t n, float* d_F,
                            elsar_stream_t stream);
elsar_status elsar_mlp_grad(const float* d_w, const uint64_t* d_knots, const uint64_t* d_x, const float* d_y,
                            uint64_t n, float* d_grad, void* d_ws, size_t ws_bytes, elsar_stream_t stream);
elsar_status elsar_mlp_splitters(const float* d_w, const uint64_t* d_knots, uint32_t log2B, uint64_t* d_t,
                                 elsar_stream_t stream);
/*
 * One Adam step of the network's training (Kingma & Ba 2015, Algorithm 1), as
 * the trainer applies it, for parity checks: with step number t >= 1, the
 * moments d_m and d_v (1517 floats each, updated in place) take the gradient
 * d_grad (1517 floats), the bias-corrected step lr * mhat / (sqrt(vhat) + 1e-8)
 * is subtracted from d_w, and the weights (not the biases) are projected onto
 * >= 0.  Decay rates 0.9 and 0.999.  FP32.  Asynchronous.
 * Errors: EINVAL (null pointers, t == 0); ECUDA.
 */
elsar_status elsar_mlp_adam(float* d_w, const float* d_grad, float* d_m, float* d_v, uint32_t t, float lr,
                            elsar_stream_t stream);

/* Bytes of the scratch area built into the library for elsar_sort_noalloc. */
#define ELSAR_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * elsar_sort for callers that cannot allocate device memory (no cudaMalloc
 * allowed or possible: plugins and callbacks whose runtime forbids it, memory
 * fully owned by another allocator, code that must not risk cudaFree's
 * device-wide synchronisation).  The paper has no counterpart; this is an
 * interface addition.  The caller passes the input and output records only;
 * scratch comes from a fixed array of ELSAR_NOALLOC_SCRATCH_BYTES (16 MiB)
 * compiled into the library, which every GPU that loads the library keeps
 * until the process exits.  The limit: elsar_workspace_size(n, p) must fit in
 * it -- about 500,000 records with the default parameters -- else the call
 * returns ELSAR_EUNSUPPORTED and allocates nothing.  The call allocates no
 * device memory itself (no cudaMalloc/cudaFree, no allocating library call).
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on one device share the one scratch
 * array and it keeps the previous call's contents (each call clears what
 * must start at zero): calls that can overlap on the GPU -- on different
 * streams, or from different threads -- race on it and must be serialised by
 * the caller.  Synchronises `stream` and reports a device-side timeout of its
 * own sort (elsar_sort, then elsar_wait on the scratch).
 */
elsar_status elsar_sort_noalloc(const void* d_in, void* d_out, uint64_t n, const elsar_params* p,
                                elsar_stream_t stream);

/*
 * Failure-detection self-test of the bounded waits that guard every TMA
 * pipeline: one CTA waits on an mbarrier phase that nothing completes while
 * one of its own 4096-byte bulk copies (from d_src, 16-byte aligned, device)
 * is in flight.  After limit_cycles (1 .. 4e9 SM clock cycles) the wait gives
 * up, the CTA raises the status word (d_word, 3 x uint32 of device memory),
 * waits (bounded) for its own copy and returns.  h_result receives the
 * 3 words: [0] bit 0 = the wait timed out, bit 1 = the in-flight copy was
 * drained; [1] the byte sum of the copied block; [2] the cycles waited
 * (saturated).  Returns ELSAR_ETIMEOUT when the wait gave up (the expected
 * outcome), ELSAR_EINVAL on bad arguments, ELSAR_ECUDA on a CUDA error.
 * Synchronises the stream.  The context stays usable afterwards.
 */
elsar_status elsar_selftest_bounded_wait(const void* d_src, void* d_word, uint64_t limit_cycles,
                                         elsar_stream_t stream, uint32_t* h_result);

/* Static description of a status code. */
const char* elsar_status_str(elsar_status s);

/* Message of the last failing call on this thread ("" if none). */
const char* elsar_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ELSAR_H */

/*
 * bp.h -- C ABI of libbp, a GB300 (sm_103a) library for the event-driven
 * spiking-network hot path of BrainPy (Wang et al., ICLR 2024, "A
 * differentiable brain simulator bridging brain simulation and brain-inspired
 * computing").
 *
 * Conventions (apply to every entry point unless its comment says otherwise)
 * ---------------------------------------------------------------------------
 * Memory.    Every array pointer is DEVICE memory owned by the caller and must
 *            stay valid until the stream work that uses it has finished.  The
 *            library allocates device memory only inside the *_create calls
 *            and frees it in the matching *_destroy.
 * Streams.   Every call is asynchronous on `stream` (a cudaStream_t; NULL is
 *            the legacy default stream) and returns after enqueueing.
 * Layout.    Vectors are dense and contiguous.  Sparse matrices are CSR with
 *            PRESYNAPTIC rows: indptr int64 [n_pre + 1] (indptr[0] = 0,
 *            non-decreasing), indices int32 [nnz] in [0, n_post).  Calls that
 *            use the post-column tile index also need each row's indices
 *            sorted ascending (canonical CSR; the JIT materialiser produces it).
 * Weights.   BP_W_HOMO (one scalar for every stored entry), BP_W_F32 or
 *            BP_W_BF16 arrays [nnz]; accumulation is always FP32, or exact
 *            int32 event counts where a call says so.
 * Output.    Outputs ACCUMULATE (y += ...) unless BP_OVERWRITE is set in flags.
 * Errors.    Every call returns a bp_status; nothing crosses the ABI as a C++
 *            exception.  Argument errors are detected on the host before any
 *            work is enqueued (BP_ERR_INVALID, nothing launched).  CUDA launch
 *            errors return BP_ERR_CUDA.  Conditions detected on the device
 *            (a bounded wait that ran out, a bounds check) set a sticky device
 *            status word, reported by bp_sync_status().  bp_last_error()
 *            returns a human-readable message for the calling thread's last
 *            failure.
 * Threads.   Calls on different streams may run concurrently if they write
 *            disjoint memory.
 * Devices.   The library keeps per-device facts for the life of the process
 *            (device addresses of its own __device__ arrays, SM count, shared
 *            memory limits).  A cudaDeviceReset (or any other teardown of a
 *            device's primary context) invalidates them: do not use the
 *            library on a device after resetting it.
 */
#ifndef BP_H
#define BP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* bp_stream_t; /* identical to cudaStream_t */

typedef enum {
    BP_OK = 0,
    BP_ERR_INVALID = 1,     /* bad argument (null pointer, size, kind) */
    BP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    BP_ERR_TIMEOUT = 3,     /* a bounded device-side wait ran out */
    BP_ERR_OOM = 4,         /* a *_create could not allocate */
    BP_ERR_UNSUPPORTED = 5, /* valid but not supported (e.g. no sm_103a device) */
    BP_ERR_DEVICE = 6       /* a device-side check failed (see bp_last_error) */
} bp_status;

typedef enum { BP_W_HOMO = 0, BP_W_F32 = 1, BP_W_BF16 = 2 } bp_wkind;

/* Weight law of a just-in-time (JIT) connectivity descriptor (Section 4.2,
 * Appendix C): homogeneous w0; uniform in [w0, w1); normal with mean w0 and
 * standard deviation w1. */
typedef enum { BP_JIT_HOMO = 0, BP_JIT_UNIFORM = 1, BP_JIT_NORMAL = 2 } bp_jit_wkind;

#define BP_OVERWRITE 1u     /* zero the output before accumulating */
#define BP_ACC_GLOBAL 2u    /* force direct atomic accumulation in L2 (no shared-memory tiles) */
#define BP_ACC_SHARED 4u    /* force shared-memory tile accumulation */
#define BP_ACC_FIXED 8u     /* float products: tile sums in 32-bit fixed point (see bp_event_csrmv) */

/* --------------------------------------------------------------------------
 * Library
 * ------------------------------------------------------------------------ */

/* Version string "bp <major>.<minor> sm_103a". Never NULL. */
const char* bp_version(void);

/* Message of the calling thread's most recent failure ("" if none). */
const char* bp_last_error(void);

/* Waits for `stream`, then reads and clears the library's sticky device
 * status word.  Returns BP_ERR_TIMEOUT / BP_ERR_DEVICE if a kernel recorded a
 * device-side failure since the last call, BP_ERR_CUDA if the stream reported
 * an error, BP_OK otherwise. */
bp_status bp_sync_status(bp_stream_t stream);

/* Shared-memory accumulator capacity (post neurons per tile) the event
 * products use for `wkind` outputs: int32 counts and FP32 sums both take 4
 * bytes per post neuron. */
int32_t bp_tile_cols(void);

/* A tile width for an index over n_post post columns: the fewest tiles of
 * at most bp_tile_cols() columns, S = ceil(n_post / bp_tile_cols()), made
 * equal, ceil(n_post / S) rounded up to a multiple of 32 (32 when
 * n_post <= 0).  The tiled products give each of the S tiles the same
 * number of CTAs, so equal tiles give every CTA the same share of a uniform
 * matrix (with full-width tiles the last one can be nearly empty). */
int32_t bp_tile_cols_for(int64_t n_post);

/* --------------------------------------------------------------------------
 * a1-a4. LIF / exponential conductance synapse / COBA step.
 * Appendix E (exponential synapse: g <- exp(-dt/tau) g, then g <- g + w per
 * delivered spike), Appendix F (tau dV/dt = -(V - V_rest) + R G with
 * G = -sum g (V - E); spike when V > V_th; V <- V_reset), Appendix N
 * Listing S6 (E/I COBA network: tau = 20 ms, tau_ref = 5 ms, E_e = 0 mV with
 * tau_e = 5 ms, E_i = -80 mV with tau_i = 10 ms, input 20 per step).
 * ------------------------------------------------------------------------ */
/* Largest refractory period, in steps, that the uint8 refractory counters
 * hold; every entry point taking bp_coba_params rejects a longer one. */
#define BP_MAX_REF_STEPS 255

typedef struct {
    double dt;              /* ms */
    double tau_m, tau_e, tau_i, tau_ref;    /* ms; round(tau_ref / dt) <= BP_MAX_REF_STEPS */
    double V_rest, V_th, V_reset, E_e, E_i; /* mV */
    double R;               /* membrane resistance */
    double I_ext;           /* constant input added every step */
    double w_e, w_i;        /* conductance increment per delivered E / I event */
} bp_coba_params;

/* Fills `p` with the COBA E/I parameters of Appendix N Listing S6
 * (dt = 0.1 ms, V_rest = V_reset = -60, V_th = -50, tau_m = 20, tau_ref = 5,
 * tau_e = 5, tau_i = 10, E_e = 0, E_i = -80, R = 1, I_ext = 20, w_e = 0.6,
 * w_i = 6.7).  Returns BP_ERR_INVALID if p is NULL. */
bp_status bp_coba_params_default(bp_coba_params* p);

/* One time step for neurons [0, n), each neuron independently:
 *   ge <- ge exp(-dt/tau_e) + dge,  gi <- gi exp(-dt/tau_i) + dgi,
 *     where dge = w_e ye[i] and dgi = w_i yi[i] if y_is_count (ye, yi are
 *     int32 event counts), else dge = ye[i], dgi = yi[i] (FP32 weighted sums);
 *     ye[i] and yi[i] are then set to 0;
 *   I = ge (E_e - V) + gi (E_i - V) + I_ext (+ I_vec[i] if I_vec != NULL),
 *     with V from before this step;
 *   if ref[i] > 0: ref[i] -= 1, V unchanged, no spike;
 *   else V <- V_inf + (V - V_inf) exp(-dt/tau_m), V_inf = V_rest + R I
 *     (exponential Euler, I held over the step); if V > V_th: spike,
 *     V <- V_reset, ref[i] <- round(tau_ref / dt).
 * The decay factors are evaluated in FP64 on the host and rounded to FP32;
 * the state arithmetic is FP32.
 * Arrays: V, ge, gi float [n]; ref uint8 [n] (refractory steps left: one
 *   byte per neuron, since this counter is read every step and the state
 *   pass is bound by memory traffic); ye, yi int32 or float [n].
 *   16-byte aligned V, ge, gi, ye, yi (I_vec, spk 16 / 4 bytes) and a
 *   4-byte aligned ref take the four-neurons-per-thread path; any alignment
 *   is accepted.
 * Outputs: spk uint8 [n] (nullable) = 1 where the neuron spiked this step;
 *   spike ids are APPENDED to spike_list int32 [n] (nullable together with
 *   n_spikes) at positions reserved by an atomic add on *n_spikes (the caller
 *   zeroes *n_spikes beforehand; the order of ids in the list is unspecified);
 *   spike_totals int64 [2] (nullable) += number of spikes among neurons
 *   [0, n_e) and [n_e, n).
 * Errors: BP_ERR_INVALID for n < 0, n_e outside [0, n], a required NULL or
 *   a refractory period round(tau_ref / dt) above 255 steps (BP_MAX_REF_STEPS,
 *   the range of the uint8 counter: 25.5 ms at dt = 0.1 ms). */
bp_status bp_lif_step(const bp_coba_params* p, int64_t n, int64_t n_e,
                      float* V, float* ge, float* gi, uint8_t* ref,
                      void* ye, void* yi, int32_t y_is_count,
                      const float* I_vec,
                      uint8_t* spk, int32_t* spike_list, int32_t* n_spikes,
                      int64_t* spike_totals, bp_stream_t stream);

/* Compacts a dense event vector (Appendix B's `events`) into a spike list:
 * appends every i with events[i] != 0 to spike_list int32 [n] at positions
 * reserved by an atomic add on *n_spikes (caller zeroes it; order
 * unspecified). */
bp_status bp_spike_compact(int64_t n, const uint8_t* events, int32_t* spike_list,
                           int32_t* n_spikes, bp_stream_t stream);

/* --------------------------------------------------------------------------
 * a5. Event-driven CSR product (Appendix B; Section 5.1 operator benchmark).
 * For every spiking presynaptic row i in spike_list[0 .. *n_spikes):
 *   for j in [indptr[i], indptr[i+1]): y[indices[j]] += w_j
 * i.e. y = W^T s with W stored presynaptic-row-major (Appendix B's listing,
 * read with the synapse index j as the column subscript).
 * w_j = data[j] (F32 / BF16) or w_homo (HOMO).  If y_is_count (HOMO only), y
 * is int32 and receives exact event counts (w_homo is not applied);
 * otherwise y is float.
 * spike_list int32 [max_spikes] with distinct ids in [0, n_pre); *n_spikes is
 * read on the device (at most max_spikes are used).
 * tile_ptr/tile_cols: optional post-column tile index from
 * bp_csr_tile_index() (NULL/0 if none); needed for shared-memory tile
 * accumulation when n_post > bp_tile_cols().
 * Accumulation order is unspecified: FP32 results are deterministic only up to
 * rounding; int32 counts are exact.
 * BP_ACC_FIXED (float y; needs a tile index on which
 * bp_csr_tile_weight_bound() has recorded the weight bound b and the column
 * count c_max): the shared-memory tile sums are 32-bit integers.  A CTA that
 * accumulates M spiking rows bounds every column of its tile by m b, with
 * m = min(M, c_max) (a column receives at most one run of entries per row),
 * takes s = 29 - e_m - e_b, where m < 2^e_m <= 2 m and b < 2^e_b <= 2 b
 * (s kept within [-126, 126]), and adds round(w_j 2^s) per event, so no
 * tile sum can overflow; the tile, times 2^-s, is then added to y in FP32.
 * Each event is off by at most 2^-(s+1) <= max(2 m b 2^-29, 2^-127)
 * absolute, the order of the worst-case rounding of an FP32 sum of the same
 * terms (the second term only for weight bounds below 2^-97 / m), and a
 * tile's sum does not depend on the order of its events.  Direct (global-atomic) accumulation ignores
 * the flag.  A tile index without a recorded bound makes the kernel record
 * BP_ERR_DEVICE (bp_sync_status) and add nothing.
 * Errors: BP_ERR_INVALID for negative sizes, NULL required pointers,
 * y_is_count with a non-HOMO kind, a tile index built for other sizes, or
 * BP_ACC_FIXED for float y without a tile index. */
bp_status bp_event_csrmv(int64_t n_pre, int64_t n_post,
                         const int64_t* indptr, const int32_t* indices,
                         const void* data, int32_t wkind, float w_homo,
                         const int32_t* spike_list, const int32_t* n_spikes, int64_t max_spikes,
                         void* y, int32_t y_is_count,
                         const int32_t* tile_ptr, int32_t tile_cols,
                         uint32_t flags, bp_stream_t stream);

/* As bp_event_csrmv, but from the dense event vector events uint8 [n_pre]
 * (the paper's form).  `workspace` is caller-owned device scratch of
 * bp_event_csrmv_dense_workspace_bytes(n_pre) bytes (spike list + count). */
size_t bp_event_csrmv_dense_workspace_bytes(int64_t n_pre);
bp_status bp_event_csrmv_dense(int64_t n_pre, int64_t n_post,
                               const int64_t* indptr, const int32_t* indices,
                               const void* data, int32_t wkind, float w_homo,
                               const uint8_t* events, void* workspace,
                               void* y, int32_t y_is_count,
                               const int32_t* tile_ptr, int32_t tile_cols,
                               uint32_t flags, bp_stream_t stream);

/* bp_event_csrmv_dense for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface convenience of this
 * library.  It computes exactly what bp_event_csrmv_dense computes (same
 * arguments, without `workspace`), keeping the compacted spike list in a
 * fixed scratch array built into the library instead of a caller-owned
 * workspace.  It is meant for code that runs inside a framework owning the
 * whole device memory pool, and for real-time loops in which cudaMalloc /
 * cudaFree could synchronise the device; it calls no allocating routine.
 * Limits: n_pre <= bp_event_csrmv_dense_noalloc_max_pre() (2^20); larger
 * inputs return BP_ERR_INVALID with a message and enqueue nothing.  The
 * scratch (about 4 MiB) exists on every GPU that loads the library until the
 * process exits.  The first call on each device looks up the scratch
 * array's device address and keeps it (see Devices above: not valid across a
 * cudaDeviceReset); make that first call before any stream capture.
 * All calls on a device share the scratch, so calls that may overlap on the
 * GPU (other streams or host threads) race and must be serialised by the
 * caller. */
int64_t bp_event_csrmv_dense_noalloc_max_pre(void);
bp_status bp_event_csrmv_dense_noalloc(int64_t n_pre, int64_t n_post,
                                       const int64_t* indptr, const int32_t* indices,
                                       const void* data, int32_t wkind, float w_homo,
                                       const uint8_t* events, void* y, int32_t y_is_count,
                                       uint32_t flags, bp_stream_t stream);

/* Post-column tile index for shared-memory accumulation.  With
 * S = ceil(n_post / tile_cols) tiles, writes tile_ptr int32
 * [n_pre * (S + 1) + 1] (bp_csr_tile_index_size entries):
 * tile_ptr[i (S+1) + s] = (first position in row i whose column is
 * >= s tile_cols) - indptr[i], for s = 0..S (so entry S is the row length),
 * and 0 in the last two entries (the bound slots of
 * bp_csr_tile_weight_bound: no bound recorded).
 * Requires sorted rows and row lengths < 2^31.  tile_cols must be a positive
 * multiple of 32 no larger than bp_tile_cols(). */
int64_t bp_csr_tile_index_size(int64_t n_pre, int64_t n_post, int32_t tile_cols);
bp_status bp_csr_tile_index(int64_t n_pre, int64_t n_post, const int64_t* indptr,
                            const int32_t* indices, int32_t tile_cols, int32_t* tile_ptr,
                            bp_stream_t stream);

/* Records in the tile index built by bp_csr_tile_index (same n_pre, n_post,
 * tile_cols) the bounds that BP_ACC_FIXED needs, in its last two entries:
 * b = the largest absolute sum of one row's entries in one column (the
 * largest |w_j| when no row repeats a column; |w_homo| for BP_W_HOMO),
 * rounded up, as FP32 bits at index n_pre (S+1); and c_max = the largest
 * number of rows with an entry in one column, as an int32 at index
 * n_pre (S+1) + 1 (bp_csr_tile_index leaves 0 in both: no bound).
 * work int32 [n_post]: caller-owned scratch (the per-column row counts),
 * overwritten; it may be NULL only when n_post = 0.  One device pass over
 * the stored entries and one over the columns; call it again after the
 * weights or the indices change.  Column indices outside [0, n_post) are
 * not counted. */
bp_status bp_csr_tile_weight_bound(int64_t n_pre, int64_t n_post, const int64_t* indptr,
                                   const int32_t* indices, const void* data, int32_t wkind,
                                   float w_homo, int32_t tile_cols, int32_t* tile_ptr,
                                   int32_t* work, bp_stream_t stream);

/* Validation of a CSR before use (the products trust their operands and do
 * not check indices on the hot path): one device pass over indices [nnz]
 * (the buffer's length) writes int64 counts out[4] = {invalid row extents
 * (indptr[i+1] < indptr[i], an extent outside [0, nnz]; plus one if
 * indptr[0] != 0 or indptr[n_pre] != nnz), entries whose index is outside
 * [0, n_post), rows not sorted ascending (bp_csr_tile_index needs sorted
 * rows), sorted rows with a repeated column}.  Rows with an invalid extent are
 * not read.  A matrix is safe for every product when the first two counts
 * are 0.  out is device memory, overwritten. */
bp_status bp_csr_check(int64_t n_pre, int64_t n_post, int64_t nnz, const int64_t* indptr, const int32_t* indices,
                       int64_t* out, bp_stream_t stream);

/* Gather ("transpose") form over the same CSR, all rows (Section 4.1: every
 * operator has reverse-mode rules; this is the product with W rather than
 * W^T):  y_pre[i] += sum_{j in row i} w_j x_post[indices[j]].
 * x_post float [n_post], y_pre float [n_pre].  With a tile index
 * (bp_csr_tile_index, sorted rows; NULL / 0 for none) x_post is staged in
 * shared memory tile by tile and each (row, tile) partial sum is added to
 * y_pre once (float atomics across tiles, so with several tiles the order of
 * the additions, and the last bits of y_pre, may vary between calls); it pays
 * when x_post is larger than the caches and rows hold a few hundred entries
 * per tile or more.  Otherwise, or with BP_ACC_GLOBAL in flags, x_post is
 * read through L1/L2 by a gather that keeps more rows in flight.
 * BP_OVERWRITE replaces y_pre instead of adding to it. */
bp_status bp_event_csrmv_t(int64_t n_pre, int64_t n_post,
                           const int64_t* indptr, const int32_t* indices,
                           const void* data, int32_t wkind, float w_homo,
                           const float* x_post, float* y_pre,
                           const int32_t* tile_ptr, int32_t tile_cols,
                           uint32_t flags, bp_stream_t stream);

/* Reverse mode of bp_event_csrmv for a loss L with dy = dL/dy (Section 4.1):
 *   dw[j] += dy[indices[j]] for every entry j of every spiking row (if dw is
 *   non-NULL; float [nnz]; each spiking row must appear once);
 *   dx_pre[i] += sum_j w_j dy[indices[j]] for every row i (if dx_pre is
 *   non-NULL; float [n_pre]: the gradient with respect to the spike vector),
 *   computed as bp_event_csrmv_t with the optional tile index (the one the
 *   forward product uses; NULL / 0 for none). */
bp_status bp_event_csrmv_bwd(int64_t n_pre, int64_t n_post,
                             const int64_t* indptr, const int32_t* indices,
                             const void* data, int32_t wkind, float w_homo,
                             const int32_t* spike_list, const int32_t* n_spikes, int64_t max_spikes,
                             const float* dy, float* dw, float* dx_pre,
                             const int32_t* tile_ptr, int32_t tile_cols,
                             bp_stream_t stream);

/* --------------------------------------------------------------------------
 * a6. Just-in-time connectivity (Section 4.2, Appendix C).
 * Row i's targets are q_0 = U_0 - 1, q_{k+1} = q_k + U_{k+1} while
 * q < n_post, with U_k = 1 + floor(x_k K / 2^32) uniform on [1, K],
 * K = ceil(2/p - 1) (at least 1), and x_k word (k mod 4) of
 * Philox4x32-10(key = seed, counter = (k div 4, i, 0, 0)).
 * Weights: HOMO w0; UNIFORM w0 + (w1 - w0) u, u = (x'_k >> 8) 2^-24 from the
 * stream-1 counter (k div 4, i, 1, 0); NORMAL w0 + w1 sqrt(-2 ln u1)
 * cos(2 pi u2) from words 2(k mod 2), 2(k mod 2)+1 of the stream-2 block
 * (k div 2, i, 2, 0), u1 = ((a >> 8) + 1) 2^-24, u2 = (b >> 8) 2^-24.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    double p;       /* connection probability in (0, 1] */
    int64_t K;      /* gap range, filled by bp_jit_desc_init */
    int32_t wkind;  /* bp_jit_wkind */
    float w0, w1;
} bp_jit_desc;

/* Fills d and computes K = ceil(2/p - 1) in FP64 (with a 1e-12 relative
 * guard so that p = a/b representing 2/(K+1) yields K).  BP_ERR_INVALID if p
 * is not in (0, 1] or wkind unknown. */
bp_status bp_jit_desc_init(bp_jit_desc* d, uint64_t seed, double p, int32_t wkind, float w0, float w1);

/* Event-driven JIT product (Appendix C listing, per-row streams):
 * y[q] += w for every target q of every row in spike_list[0 .. *n_spikes).
 * y int32 exact counts if y_is_count (HOMO only) else float. */
bp_status bp_jitconn_event_mv(const bp_jit_desc* d, int64_t n_pre, int64_t n_post,
                              const int32_t* spike_list, const int32_t* n_spikes, int64_t max_spikes,
                              void* y, int32_t y_is_count, uint32_t flags, bp_stream_t stream);

/* Reverse mode with respect to the spike vector (weights are static, so
 * there is no weight gradient, Section 4.2): dx_pre[i] += sum over row i's
 * targets q of w dy[q], for all rows i. */
bp_status bp_jitconn_event_mv_bwd(const bp_jit_desc* d, int64_t n_pre, int64_t n_post,
                                  const float* dy, float* dx_pre, bp_stream_t stream);

/* Non-event JIT product with a dense vector (Section 5.2, mv_prob_uniform /
 * mv_prob_normal): y_post[q] += w x_pre[i] for every target q of every row i. */
bp_status bp_jitconn_mv(const bp_jit_desc* d, int64_t n_pre, int64_t n_post,
                        const float* x_pre, float* y_post, uint32_t flags, bp_stream_t stream);

/* Materialises the JIT matrix as CSR.  First call with indices == NULL: writes
 * indptr int64 [n_pre + 1] (row lengths, then an in-place prefix sum).  Then
 * call again with indices int32 [indptr[n_pre]] (and data float/bf16 [nnz] if
 * data_kind != BP_W_HOMO) to fill the rows (sorted ascending). */
bp_status bp_jit_materialize_csr(const bp_jit_desc* d, int64_t n_pre, int64_t n_post,
                                 int64_t* indptr, int32_t* indices, void* data, int32_t data_kind,
                                 bp_stream_t stream);

/* Projection seed of the E/I network: output `projection` (0 = E rows,
 * 1 = I rows) of SplitMix64 started at net_seed (Steele et al. 2014). */
uint64_t bp_projection_seed(uint64_t net_seed, int32_t projection);

/* --------------------------------------------------------------------------
 * a7/a8. COBA E/I network: step and simulate (Appendix N Listing S6).
 * Neurons [0, n_e) are excitatory, [n_e, n) inhibitory.  Each step is the
 * bp_lif_step update followed by the delivery of this step's spikes: E rows
 * into ye, I rows into yi (one merged conductance per neuron and synapse
 * type, Section 4.3 AlignPost), consumed by the next step.  The event
 * accumulators are double-buffered ([2n] each): step t reads and clears
 * elements [(t mod 2) n, (t mod 2 + 1) n) and delivers into the other half,
 * which lets one kernel do both.
 * Synaptic delay (Appendix D: a projection retrieves the presynaptic spikes
 * after its delay): with delay_e = d > 0 the E spikes of step t act at step
 * t + 1 + d instead of t + 1 (likewise delay_i for the I spikes).  The spike
 * ids of each step are kept in a ring of D + 2 lists, D = max(delay_e,
 * delay_i), in the caller's delay_buf: int32 [(D + 2) (n + 1)], the D + 2
 * counts followed by D + 2 lists of n ids.  Step t appends its spikes to
 * list t mod (D + 2) and, over all CTAs, delivers the rows of the spikes of
 * step t - d into the accumulator half that step t + 1 reads; a projection
 * with delay 0 delivers its own spikes as above.
 * AlignPre form (align = BP_ALIGN_PRE, Appendix D): instead of one merged
 * conductance per postsynaptic neuron, one synaptic trace per presynaptic
 * neuron, s_i <- s_i a + z_i (a = exp(-dt/tau_e) on E rows, exp(-dt/tau_i) on
 * I rows, z the previous step's spike flags), and every step the
 * conductances are recomputed through the connection matrix, g_e = W_E^T s
 * (times w_e for homogeneous weights), g_i likewise.  For these exponential
 * synapses it is the same dynamics as AlignPost at the cost of a full
 * product per step; each step is two launches (trace + product, then the
 * neurons).  It needs `trace` [n] (initially 0), `spk` (the flags are its
 * input), float accumulators (ye, yi [2n] float whatever the weights) and no
 * delay; totals[2] counts each step's synaptic events when the next step
 * consumes them.
 * ------------------------------------------------------------------------ */
enum { BP_CONN_CSR = 0, BP_CONN_JIT = 1 };

typedef struct {
    int64_t n, n_e;
    bp_coba_params coba;
    int32_t conn_kind;              /* BP_CONN_CSR or BP_CONN_JIT */
    /* BP_CONN_CSR: one CSR over all n presynaptic rows (row i < n_e: E
     * projection row i; row i >= n_e: I projection row i - n_e). */
    const int64_t* indptr;
    const int32_t* indices;
    const void* data;               /* NULL or wkind == BP_W_HOMO: weights w_e / w_i, int32 counts */
    int32_t wkind;
    const int32_t* tile_ptr;        /* optional, see bp_csr_tile_index */
    int32_t tile_cols;
    /* BP_CONN_JIT: homogeneous rows with seeds bp_projection_seed(seed, 0/1) */
    uint64_t seed;
    double p;
    /* state, device, caller-owned */
    float* V;                       /* [n] */
    float* ge;                      /* [n] */
    float* gi;                      /* [n] */
    uint8_t* ref;                   /* [n] refractory steps left (see bp_lif_step) */
    void* ye;                       /* [2n] int32 counts (homogeneous) or float sums, two halves */
    void* yi;                       /* [2n] */
    int32_t* spike_list;            /* [n] nullable: spike ids of the last step (order unspecified) */
    int32_t* n_spikes;              /* [2] with spike_list: the last step t's count is n_spikes[t mod 2] */
    int64_t* totals;                /* [4] cumulative: spikes E, spikes I, synaptic events, steps */
    uint8_t* spk;                   /* [n] nullable: spike flags of the last step */
    int32_t delay_e, delay_i;       /* synaptic delays in steps, 0 .. 65535 (0 = next step) */
    int32_t* delay_buf;             /* [(D + 2)(n + 1)] when a delay is > 0 (see above), else NULL */
    int32_t align;                  /* BP_ALIGN_POST (default) or BP_ALIGN_PRE */
    float* trace;                   /* [n] presynaptic traces for BP_ALIGN_PRE, else NULL */
} bp_net_desc;

enum { BP_ALIGN_POST = 0, BP_ALIGN_PRE = 1 };

typedef struct bp_net bp_net;

/* Validates `desc`, copies it, derives the decay factors and JIT seeds.
 * Allocates the handle and a 32-byte device control block (step counter,
 * record target); the CUDA graph of bp_simulate is built on its first call.
 * *out receives the handle. */
bp_status bp_network_create(const bp_net_desc* desc, bp_net** out);

/* Zeroes the counters (n_spikes, totals), both halves of the event
 * accumulators and the delay ring's counts, and restarts the step count at
 * 0. */
bp_status bp_network_reset_counters(bp_net* net, bp_stream_t stream);

/* One time step (a1-a5/a6 above). */
bp_status bp_network_step(bp_net* net, bp_stream_t stream);

/* Checkpoint / resume.  The network's state lives in the caller's buffers
 * named in bp_net_desc (V, ge, gi, ref, both halves of ye and yi, the delay
 * ring, the AlignPre traces, spk, n_spikes and totals); the library keeps one
 * more number, the count of steps since the last reset, which selects the
 * accumulator half, the counter slot and the delay-ring slot of the next
 * step.  To checkpoint, copy those buffers and read the count; to resume (on
 * this or a new network with the same desc layout), write the buffers back
 * and set the count.  bp_network_step_count returns the count of the steps
 * enqueued so far (-1 for a NULL handle); bp_network_set_step_count enqueues
 * the new count on `stream` (step >= 0). */
int64_t bp_network_step_count(const bp_net* net);
bp_status bp_network_set_step_count(bp_net* net, int64_t step, bp_stream_t stream);

/* T steps, launched as CUDA graphs on `stream`: T is split into 64-step
 * chunks and a shorter remainder; the graph of each length is captured once
 * per parity of the starting step count, on a private stream, on first use
 * and cached with the network.  record int32 [T][2] (nullable) receives the
 * E and I spike counts of each step. */
bp_status bp_simulate(bp_net* net, int64_t T, int32_t* record, bp_stream_t stream);

/* Captures (if not cached yet) and uploads to the device, on `stream`, the
 * graphs that bp_simulate(net, T, ...) launches, without running any step:
 * a later bp_simulate of T steps then spends no host time on capture or
 * instantiation and its first launch no time on the upload. */
bp_status bp_simulate_prepare(bp_net* net, int64_t T, bp_stream_t stream);

/* Population statistics in FP64 on the device (a8): out double [4] =
 * {rate of all neurons, E rate, I rate (Hz), synaptic events per step}, from
 * the int64 totals accumulated since the last reset. */
bp_status bp_network_stats(bp_net* net, double* out, bp_stream_t stream);

/* Sparse form of a checkpointed event accumulator (between steps the live
 * half holds the deliveries of the last step's spikes, mostly zero).
 * bp_words_compact: the nonzero 32-bit words of x [n] (int32 counts or FP32
 * bits; -0.0f counts as nonzero) into idx int32 [n] and val uint32 [n]
 * (capacity n, caller-owned), their number into *count (device int32, set
 * by the call); pairs are in no particular order.  bp_words_scatter:
 * x[idx[k]] = val[k] for k < count (host count; indices outside [0, n)
 * are skipped); the other words of x are left as they are.  n < 2^31. */
bp_status bp_words_compact(const void* x, int64_t n, int32_t* idx, uint32_t* val, int32_t* count,
                           bp_stream_t stream);
bp_status bp_words_scatter(const int32_t* idx, const uint32_t* val, int64_t count, void* x, int64_t n,
                           bp_stream_t stream);

bp_status bp_network_destroy(bp_net* net);

/* --------------------------------------------------------------------------
 * a9. Batched networks: many independent COBA E/I networks of uneven sizes
 * (the "parameter explorations" of Section 3), each with its own seed and
 * either JIT connectivity (probability p, default 80/n) or stored CSR rows,
 * homogeneous w_e / w_i, advanced together by one persistent kernel in which
 * a CTA owns whole networks (no inter-CTA synchronisation), its time loop
 * captured in a CUDA graph.  The per-step arithmetic is the one of
 * bp_network_step; a network of the batch follows the trajectory the
 * single-network path computes for it.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_nets;
    const int64_t* n;       /* HOST [n_nets] neurons per network, each in [1, 56320] */
    const int64_t* n_e;     /* HOST [n_nets] nullable: default 4n/5 (each population < 65536) */
    const uint64_t* seed;   /* HOST [n_nets] network seeds (projection seeds derived as in bp_projection_seed) */
    const double* p;        /* HOST [n_nets] nullable: default 80/n */
    bp_coba_params coba;    /* shared by every network */
    /* device state, caller-owned, concatenated: network b occupies
     * [off_b, off_b + n_b) with off_b from bp_batch_layout; padding entries
     * are never simulated.  V, ge, gi must be 16-byte and ref 4-byte aligned
     * (four neurons per access; BP_ERR_INVALID otherwise). */
    float* V;
    float* ge;
    float* gi;
    uint8_t* ref;           /* refractory steps left (see bp_lif_step) */
    int64_t* totals;        /* device [n_nets][4]: spikes E, spikes I, events, steps (accumulated) */
    /* Stored connectivity (both NULL: JIT rows from the seeds): one CSR over
     * the padded concatenated layout, device memory.  Row off_b + i holds the
     * targets of neuron i of network b (E rows i < n_e_b, I rows after) as
     * indices local to network b, strictly increasing, in [0, n_b); padding
     * rows are empty.  Validated by bp_batch_create (BP_ERR_INVALID
     * otherwise); must stay valid and unchanged while the batch exists. */
    const int64_t* indptr;  /* [padded_total + 1] */
    const int32_t* indices; /* [indptr[padded_total]] */
} bp_batch_desc;

typedef struct bp_batch bp_batch;

/* Offsets of the concatenated layout: offsets[b] for b < n_nets (host,
 * nullable) and offsets[n_nets] = the total length returned (each network
 * padded to a multiple of 4 neurons).  Returns -1 on bad arguments. */
int64_t bp_batch_layout(int32_t n_nets, const int64_t* n, int64_t* offsets);

/* Validates (for stored rows: one synchronous device pass over them), packs
 * the networks into one bin per SM (longest first, bounded by shared memory)
 * and allocates the device tables, the event-count spill buffer and the
 * autotuner's snapshot.  Pending event counts start at zero.  Initial
 * tuning: 1024 threads, 8 lanes per stored row / 32 per JIT row, one CTA per
 * SM. */
bp_status bp_batch_create(const bp_batch_desc* desc, bp_batch** out);

/* Bins (CTAs), CTA size in use and padded length of the layout. */
bp_status bp_batch_info(const bp_batch* b, int32_t* bins, int32_t* threads, int64_t* padded_neurons);

/* The tuning in use: CTA size, lanes that walk one delivered row (stored
 * rows 4, 8, 16 or 32; JIT rows 16 or 32), CTAs (bins) per SM of the packing
 * (1, 2 or 4; a bin holds at most 56 320, 27 648 or 13 312 neurons), and 1 if
 * the rows are stored (0: JIT).  Any pointer may be NULL. */
bp_status bp_batch_tuning(const bp_batch* b, int32_t* threads, int32_t* lanes_per_row, int32_t* ctas_per_sm,
                          int32_t* stored_rows);

/* Sets the tuning (values as above; re-packs when ctas_per_sm changes;
 * BP_ERR_INVALID if a network does not fit the bins).  Synchronous. */
bp_status bp_batch_set_tuning(bp_batch* b, int32_t threads, int32_t lanes_per_row, int32_t ctas_per_sm);

/* Zeroes the pending event counts and the totals. */
bp_status bp_batch_reset_counters(bp_batch* b, bp_stream_t stream);

/* T steps of every network (a CUDA graph per distinct T, cached). */
bp_status bp_batch_simulate(bp_batch* b, int64_t T, bp_stream_t stream);

/* Captures (if not cached yet) and uploads, on `stream`, the graph of a
 * T-step bp_batch_simulate without running it.  A change of tuning drops the
 * cached graphs. */
bp_status bp_batch_prepare(bp_batch* b, int64_t T, bp_stream_t stream);

/* Autotuner: from a snapshot of the current state, times probe_steps steps
 * of every feasible tuning -- CTA size (256, 512, 1024 threads) x lanes per
 * delivered row x CTAs per SM (packings into 1, 2 or 4 bins per SM where
 * every network fits and the CTAs can share an SM) -- then restores the
 * state, keeps the fastest (see bp_batch_tuning) and returns its CTA size in
 * *chosen_threads (nullable).  Every tuning computes the same trajectories.
 * Synchronises `stream`. */
bp_status bp_batch_autotune(bp_batch* b, int32_t probe_steps, int32_t* chosen_threads, bp_stream_t stream);

bp_status bp_batch_destroy(bp_batch* b);

/* --------------------------------------------------------------------------
 * a10. Differentiable recurrent spiking network and its BPTT adjoint
 * (Appendix I: LIF recurrent layer with exponential synaptic current, leaky
 * readout, cross-entropy on the readout, surrogate-gradient training;
 * Section 4.1: every operator has a reverse-mode rule).  Per batch element,
 * t = 1..T, starting from I = V = y = 0 and no spikes:
 *   I_t  = a_s I_{t-1} + W_rec^T z_{t-1} + W_in^T u_t     (a_s = exp(-dt/tau_s))
 *   Vp_t = a_m V_{t-1} + (1 - a_m)(V_rest + R I_t)        (exponential Euler)
 *   z_t  = [Vp_t > V_th];  V_t = z_t ? V_reset : Vp_t      (reset detached)
 *   y_t  = a_o y_{t-1} + dt (W_out^T z_t + b_out);  m = mean_t y_t
 * Gradients use the surrogate dz/dVp ~ slope s(slope x)(1 - s(slope x)),
 * x = Vp - V_th, s the logistic function (BP_SG_SIGMOID), or the ReLU
 * surrogate of Appendix I, max(0, sg_alpha (sg_width - |x|)) (BP_SG_RELU).
 * With lambda_v > 0 the loss includes the voltage regulariser of Appendix I
 * (training methods), on the potential before reset and averaged over the
 * batch like the cross-entropy:
 *   L_v = (lambda_v / B) sum_b sum_t sum_i [max(Vp - v_hi, 0)^2 + max(v_lo - Vp, 0)^2]
 * (bp_snn_forward accumulates it, bp_snn_reg_loss adds it to the loss and
 * bp_snn_backward includes its gradient).  W_rec is CSR with presynaptic rows (event-driven
 * delivery of z_{t-1}); its stored values are FP32 or BF16, all arithmetic is
 * FP32.  Checkpoints every ckpt_every steps; the backward pass recomputes
 * each segment from its checkpoint, replaying the spikes the forward
 * recorded.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t B, T, n_in, n_rec, n_out;  /* n_in, n_rec <= 4096, n_out <= 64 */
    double dt, tau_m, tau_s, tau_o;    /* ms */
    double V_rest, V_reset, V_th, R, slope;
    int32_t ckpt_every;                /* K >= 1; 0 = a single segment (store everything) */
    const float* W_in;                 /* [n_in][n_rec] */
    const int64_t* indptr;             /* [n_rec + 1] */
    const int32_t* indices;            /* [nnz] */
    const void* w_rec;                 /* [nnz] FP32 or BF16 */
    int32_t w_rec_kind;                /* BP_W_F32 or BP_W_BF16 */
    const float* W_out;                /* [n_rec][n_out] */
    const float* b_out;                /* [n_out] */
    int64_t nnz;                       /* number of stored recurrent weights (= indptr[n_rec]) */
    int32_t surrogate;                 /* BP_SG_SIGMOID (uses slope) or BP_SG_RELU */
    double sg_alpha, sg_width;         /* ReLU surrogate height factor and half-width (> 0) */
    double lambda_v;                   /* voltage regulariser strength (>= 0; 0 = off) */
    double v_hi, v_lo;                 /* regulariser bounds, v_lo < v_hi */
} bp_snn_desc;

enum { BP_SG_SIGMOID = 0, BP_SG_RELU = 1 };

/* dt = 1 ms, tau_m = 20, tau_s = 100, tau_o = 20 ms, V_rest = V_reset = 0,
 * V_th = 1, R = 1, slope = 4, ckpt_every = 100, F32 recurrent weights,
 * logistic surrogate (sg_alpha = 0.3, sg_width = 1 for the ReLU one),
 * lambda_v = 0, v_hi = 0.4, v_lo = -2; sizes and pointers zero. */
bp_status bp_snn_desc_default(bp_snn_desc* d);

/* Device workspace (bytes, 256-byte aligned) shared by forward and backward:
 * checkpoints, the recorded spike bits of every step, one segment of
 * potentials, Ibar of every step with the operands of the weight-gradient
 * contraction (dW_in and dw_rec are one tensor-core contraction over batch
 * and time, as bp_spike_outer computes it), the readout-gradient partials of
 * each batch element (summed over the batch in a fixed order) and the
 * recurrent weights in the fixed-point form the forward delivers them in.
 * Every gradient is reproducible bit for bit.  0 for an invalid desc. */
size_t bp_snn_workspace_bytes(const bp_snn_desc* d);

/* Forward pass over T steps: u uint8 [B][T][n_in] (input spikes), m float
 * [B][n_out] (mean readout).  Fills the workspace for bp_snn_backward. */
bp_status bp_snn_forward(const bp_snn_desc* d, const uint8_t* u, float* m, void* workspace, bp_stream_t stream);

/* Adjoint of one step of the LIF layer above, neuron by neuron (the update
 * bp_snn_backward applies inside its time loop): with x = Vp - V_th and the
 * desc's surrogate,
 *   Vpbar = Vbar (1 - z) + zbar surrogate(x)
 *           + (lambda_v / B) (2 max(Vp - v_hi, 0) - 2 max(v_lo - Vp, 0))
 *   Ibar = (1 - a_m) R Vpbar + a_s Ibar_next,   Vbar_prev = a_m Vpbar
 * (reset detached; the regulariser term only when lambda_v > 0, B taken as 1
 * when it is not positive).  Arrays [n]: Vp (potential before reset at step
 * t), z (uint8 spike flags of step t), Vbar = dL/dV_t, zbar = dL/dz_t,
 * Ibar_next = dL/dI_{t+1}; outputs Ibar = dL/dI_t, Vbar_prev = dL/dV_{t-1}.
 * Only the constants of `d` are used (dt, tau_m, tau_s, V_th, R, the
 * surrogate and regulariser fields, B). */
bp_status bp_lif_step_bwd(const bp_snn_desc* d, int64_t n, const float* Vp, const uint8_t* z, const float* Vbar,
                          const float* zbar, const float* Ibar_next, float* Ibar, float* Vbar_prev,
                          bp_stream_t stream);

/* Mean over the batch of the cross-entropy of softmax(m_b) with label_b
 * (labels int64 [B]), written to loss[0], and its gradient g_m = dL/dm
 * [B][n_out].  FP32 (max-subtracted log-sum-exp; the batch mean a
 * compensated sum in batch order). */
bp_status bp_snn_loss(int32_t B, int32_t n_out, const float* m, const int64_t* labels, float* loss, float* g_m,
                      bp_stream_t stream);

/* Adds the voltage regulariser L_v accumulated by the last bp_snn_forward
 * with this desc and workspace to loss[0] (FP32 compensated sums: per thread,
 * then a fixed tree over the CTA, then the batch elements in order, so the
 * result is reproducible).  Does nothing when lambda_v = 0. */
bp_status bp_snn_reg_loss(const bp_snn_desc* d, const void* workspace, float* loss, bp_stream_t stream);

/* Weight gradient of a spike-driven dense connection (Section 3.1: for
 * y_k = W^T x_k with binary x_k the reverse-mode rule gives
 * dW = sum_k x_k dy_k^T):
 *   out[m][n] += sum_{k < K} [x[k][m] != 0] delta[k][n]
 * x uint8 [K][M] (row-major; any non-zero byte is a spike), delta float
 * [K][N], out float [M][N] (BP_OVERWRITE: out = the sum).  Computed on the
 * tensor cores (tcgen05 BF16 MMAs, FP32 accumulation): delta enters as two
 * BF16 terms, hi = bf16(delta) and lo = bf16(delta - hi), so each product
 * is exact to 2^-17 relative and the sum is FP32.  The same inputs give the
 * same result bit for bit.  work: device workspace of at least
 * bp_spike_outer_workspace(K, M, N) bytes, 1024-byte aligned, owned by the
 * caller (the call packs both operands into it).  K <= 2^31 - 1 and
 * M N < 2^31 (BP_ERR_INVALID otherwise).  K, M or N
 * zero: nothing to add (BP_OVERWRITE still zeroes out). */
size_t bp_spike_outer_workspace(int64_t K, int32_t M, int32_t N);
bp_status bp_spike_outer(const uint8_t* x, const float* delta, int64_t K, int32_t M, int32_t N, float* out,
                         uint32_t flags, void* work, size_t work_bytes, bp_stream_t stream);

/* Backward pass (BPTT with checkpointed recomputation) for an upstream
 * gradient g_m = dL/dm [B][n_out], after bp_snn_forward with the same desc,
 * inputs and workspace.  ACCUMULATES dW_in [n_in][n_rec], dw_rec [nnz] (one
 * gradient per stored recurrent weight), dW_out [n_rec][n_out] and
 * db_out [n_out]. */
bp_status bp_snn_backward(const bp_snn_desc* d, const uint8_t* u, const float* g_m, void* workspace, float* dW_in,
                          float* dw_rec, float* dW_out, float* db_out, bp_stream_t stream);

/* --------------------------------------------------------------------------
 * Measurement kernels (roofline denominators).  The paper has no counterpart:
 * these give the roofs that bound this library's kernels where HBM bandwidth
 * does not (the JIT rows' integer arithmetic, scattered L2 reductions, and the
 * state pass of networks whose state stays in L2).  Each call enqueues one
 * kernel on `stream`; the caller times it (CUDA events) and divides the work
 * stated below by the time.
 * ------------------------------------------------------------------------ */

/* Philox-only draw rate: bp_roof_philox_threads() threads each compute
 * blocks_per_thread Philox4x32-10 blocks (key `seed`, counters distinct per
 * thread and block; 4 32-bit words per block, the draws of Section 4.2's
 * JIT rows) and write one word each to sink uint32 [bp_roof_philox_threads()]
 * (device).  Work: 4 x threads x blocks_per_thread words. */
int64_t bp_roof_philox_threads(void);
bp_status bp_roof_philox(int64_t blocks_per_thread, uint64_t seed, uint32_t* sink, bp_stream_t stream);

/* Scattered-reduction rate: bp_roof_l2_red_threads() threads each add 1 to
 * per_thread pseudo-random elements of y int32 [n] (device, n in [1, 2^31))
 * with the keep-in-L2 hint of the event delivery.  Work: threads x per_thread
 * reductions (y receives that many counts in total). */
int64_t bp_roof_l2_red_threads(void);
bp_status bp_roof_l2_red(int32_t* y, int64_t n, int64_t per_thread, bp_stream_t stream);

/* Copy bandwidth: `reps` passes of dst[0, bytes) = src[0, bytes) (device,
 * 16-byte aligned, bytes a multiple of 16).  With 2 x bytes well below the
 * L2 size the buffers stay in L2 and the rate (2 x bytes x reps / time) is
 * the L2-resident copy bandwidth; above it, the HBM copy bandwidth. */
bp_status bp_roof_copy(const void* src, void* dst, int64_t bytes, int32_t reps, bp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* BP_H */

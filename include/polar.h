/*
 * polar.h -- C ABI of the GB300 successive-cancellation (SC) polar decoder.
 *
 * The method is the error-correction step of QKD with polar codes, after
 * Jouguet & Kunz-Jacques (arXiv 1204.5882):
 *   - syndrome form (Sec. 1): Alice sends no codeword; Bob holds channel
 *     LLRs of Alice's string x and Alice reveals u_F = (x G_N)_F, the
 *     values of the frozen positions of u = x G_N;
 *   - frozen set = the least reliable bit-channels (Sec. 3);
 *   - recursive SC decoding with the phi-based LLR update (Sec. 4).
 *
 * Conventions shared by every entry point:
 *   - N = 2^log2n, 1 <= log2n <= 27.  Transform x = u F^{(x)n} with
 *     F = [[1,0],[1,1]] in natural order (no bit reversal); it is its own
 *     inverse over GF(2).
 *   - Bit vectors are packed little-endian in uint32 words: bit i of a
 *     frame is bit (i % 32) of word (i / 32).  A frame of N bits takes
 *     max(1, N/32) words; frames of a batch are contiguous.
 *   - LLR L = ln P(y|x=0)/P(y|x=1).  An information bit decides 1 iff
 *     L < 0 (both +0.0 and -0.0 decide 0).
 *   - Every pointer named *_dev is device memory owned by the caller.  The
 *     library owns frozen-set objects, its per-stream scratch workspace and
 *     its cached CUDA graphs.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Decode and map calls are asynchronous and stream-ordered;
 *     the outputs are ready when the stream reaches that point.
 *   - Errors: a negative polar_status; nothing is thrown across the ABI.
 *     Argument errors are detected on the host before any launch.
 *     POLAR_ECUDA reports a CUDA error (polar_last_error_string() has the
 *     CUDA text).
 *
 * Thread safety: calls on different streams may run from different host
 * threads; frozen-set objects are read-only after construction.
 */
#ifndef POLAR_GB300_H
#define POLAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    POLAR_OK = 0,
    POLAR_EINVAL = -1,     /* bad argument (size, pointer, enum, alignment) */
    POLAR_ENOMEM = -2,     /* host or device allocation failed */
    POLAR_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    POLAR_ETIMEDOUT = -4,  /* a bounded device-side wait expired */
    POLAR_EBUSY = -5,      /* admission refused (server) */
    POLAR_ENOTFOUND = -6,  /* unknown ticket or option */
    POLAR_ECANCELED = -7,  /* request withdrawn before it ran (server) */
    POLAR_EFAULT = -8,     /* guard mode: a kernel wrote outside its scratch */
    POLAR_PENDING = 1      /* request still running (server poll) */
} polar_status;

typedef enum { POLAR_BSC = 0, POLAR_BIAWGN = 1 } polar_channel;
typedef enum { POLAR_F_MINSUM = 0, POLAR_F_EXACT = 1 } polar_fkind;
typedef enum { POLAR_FP32 = 0, POLAR_FP16 = 1, POLAR_INT8 = 2 } polar_prec;

typedef struct polar_frozen_set polar_frozen_set;

/* ------------------------------------------------------------------ misc */

/* Text for a polar_status value (static storage). */
const char *polar_strerror(int status);

/* CUDA error text of the last POLAR_ECUDA on this host thread ("" if none). */
const char *polar_last_error_string(void);

/* Process-wide tuning knobs, by name.  Returns POLAR_ENOTFOUND for an
 * unknown key, POLAR_EINVAL for a value out of range.  Keys:
 *   "subtree_log2"  t, log2 of the leaves one CTA decodes in shared memory
 *                   (5..14; default 14); levels above t stream through HBM.
 *   "persist_log2"  the same for the persistent decoder and the persistent
 *                   server (5..14; default 13, two CTAs per SM).
 *   "shortcuts"     1 = rate-0 / rate-1 node shortcuts (default), 0 = none.
 *   "graphs"        1 = replay batch launch sequences as CUDA graphs
 *                   (default), 0 = launch every kernel eagerly.
 *   "plain"         1 = the plain per-frame baseline: frames decoded one
 *                   after another, no shortcuts, no graphs; 0 (default).
 *   "profile"       time every kernel group with CUDA events (see
 *                   polar_profile_read): 1 = a one-off CUDA-graph replay of
 *                   the batch's schedule with an event-record node around
 *                   each group (device times without host launch gaps; eager
 *                   when "graphs" is 0 or the stream is the legacy default
 *                   or capturing), 2 = eager launches; 0 (default) = off.
 *   "autotune"      1 = use the schedule polar_autotune found for a batch
 *                   shape (default); 0 = ignore tuned entries.
 *   "fuse"          1 = each streamed f/g step and the f steps continuing it
 *                   run as one fused column kernel (default); 0 = one launch
 *                   per step.
 *   "split_log2"    s > t: every node of 2^s leaves (not rate 0) is decoded
 *                   by one launch of one CTA per frame, which runs the f / g
 *                   steps of the levels s..t+1 itself (over the frame's rows
 *                   of the scratch workspace, staged through shared memory)
 *                   and then its subtrees; the levels above s stay streamed
 *                   launches.  0 (default) = no such units; 6..27, ignored
 *                   when s <= t, s >= log2 N or shortcuts are off.  Results
 *                   do not depend on it (every step is the same operation
 *                   with the same storage rounding).
 *   "prologue"      1 = with float32 storage, each subtree kernel performs
 *                   the streamed step that produces its input (the f or g
 *                   from level t + 1) while loading, instead of a separate
 *                   launch; 0 (default).  Results do not depend on it.
 *   "int8_target"   INT8 storage: the per-frame scale is the power of two
 *                   2^rint(log2(target / mean|L|)) (mean in double over the
 *                   frame's channel LLRs); 1..64, default 8.
 *   "pdl"           1 = launch the kernels of a decode with programmatic
 *                   dependent launch: each waits for its predecessor's
 *                   completion on the device while its own launch overlaps
 *                   the predecessor's tail; 0 (default) = plain stream order
 *                   (graph replays already keep the gaps short; PDL measured
 *                   no faster).  Results do not depend on it.
 *   "persistent"    how polar_sc_decode_batch runs float32 batches: 0 =
 *                   always as launched groups of equally strided frames;
 *                   1 (default) = in one persistent launch
 *                   (polar_sc_decode_persistent) when the batch holds more
 *                   than one such group; 2 = always persistent.
 *   "guard"         debugging aid, 0 (default) or 1: the library's scratch
 *                   workspaces carry 64 KB guard zones of a fixed byte
 *                   pattern before and right after the bytes each decode
 *                   uses; polar_sc_decode, _many, _batch and _persistent
 *                   then wait for their stream and check both zones,
 *                   returning POLAR_EFAULT (the offset in
 *                   polar_last_error_string) if a kernel wrote outside its
 *                   scratch.  Off, nothing is added or checked.
 * Environment: POLAR_LOG set to anything but "" or "0" (read once) prints
 * "[polar] ..." diagnostics on stderr -- frozen-set constructions (K, time),
 * autotune choices, tune-cache files and server launches.
 */
int polar_config_set(const char *key, long value);

/* Debugging aid, no counterpart in the paper.  Guard-mode self-test:
 * overwrite one byte of the trailing guard zone of the
 * scratch workspace that the last decode on `stream` used (a write inside
 * the allocation), so that the next checked decode on that stream must
 * report POLAR_EFAULT.  POLAR_ENOTFOUND if that stream has no guarded
 * workspace. */
int polar_debug_spoil_guard(void *stream);
int polar_config_get(const char *key, long *value);

/* Cumulative number of kernels this library has launched in this process,
 * kernels inside replayed CUDA graphs included. */
uint64_t polar_kernel_launches(void);

/* Per-kind kernel timing, for profiling.  While the "profile" option is
 * set, decode and map calls bracket every kernel group with CUDA events on
 * the launching stream (inside a one-off graph replay, or eagerly).
 * polar_profile_read synchronises the recorded events and returns, for one
 * kind ("llr", "stream_f", "stream_g", "subtree", "rate0", "chain",
 * "persist"), the summed device time in ms, the number of launches and the
 * algorithmic bytes those launches move (inputs read once, outputs written
 * once).  polar_profile_reset discards
 * what was recorded.  Any pointer may be NULL. */
int polar_profile_read(const char *kind, double *total_ms, uint64_t *launches,
                       double *alg_bytes);
void polar_profile_reset(void);

/* --------------------------------------------------------- construction */

/* Frozen set of the code of length N = 2^log2n and K = floor(rate * N)
 * information bits for channel `ch` with parameter `param` (crossover
 * probability p of the BSC, noise variance sigma^2 of the BI-AWGN channel
 * with +-1 inputs).  Sec. 3: the N-K least reliable bit-channels are frozen.
 * Reliability: Bhattacharyya recursion Z- = 2Z - Z^2, Z+ = Z^2 from
 * Z0 = 2 sqrt(p(1-p)) (BSC); Gaussian approximation of density evolution
 * m0 = 2/sigma^2, m+ = 2m, m- = phi^-1(1 - (1 - phi(m))^2),
 * P_e = Q(sqrt(m/2)) (BI-AWGN).  Equal reliabilities freeze the lower index
 * first.  Runs on the host in double precision; the device copy is made on
 * first use.  *out receives a library-owned object (free with
 * polar_frozen_set_free).  EINVAL: log2n outside 1..27, p outside (0, 0.5),
 * sigma^2 <= 0, rate outside [0, 1], out == NULL. */
int polar_build_frozen_set(uint32_t log2n, polar_channel ch, double param,
                           double rate, polar_frozen_set **out);

/* As polar_build_frozen_set, with K chosen by Sec. 3's rule instead of a
 * rate: the largest K whose most reliable bit-channels have sum_i P_e,i <=
 * sum_pe_max, with P_e,i = Z_i (BSC: the Bhattacharyya parameter, an upper
 * bound on the error probability, loose at high rates) or the Gaussian-
 * approximation estimate Q(sqrt(m_i / 2)) (BI-AWGN: an estimate, not a
 * bound).  EINVAL as polar_build_frozen_set, or sum_pe_max < 0. */
int polar_build_frozen_set_sum(uint32_t log2n, polar_channel ch, double param,
                               double sum_pe_max, polar_frozen_set **out);

/* The construction of polar_build_frozen_set (rate > 0) or of
 * polar_build_frozen_set_sum (rate = 0, with sum_pe_max), computed on the
 * current CUDA device in double precision (Sec. 3: frozen bits are the least
 * reliable bit-channels; on the device a new code costs milliseconds, which
 * makes it the request server's cache miss): each polarisation level is one
 * launch, the bit-channels
 * are ranked by a stable radix sort of (reliability, index) with the lower
 * index frozen first on equal reliability, and Sec. 3's rule takes a prefix
 * sum of P_e along the ranking.  Stream-ordered on `stream`, synchronous on
 * return (the mask is read back to the host; the device copy stays resident
 * for decodes on this device).  Takes about 2N * 40 bytes of device memory
 * while it runs.  The device's exp / log / pow round differently from the
 * host's in the last bit, so the set can differ from the host construction
 * only at bit-channels whose reliability is within rounding of the K-th one
 * (and, with the sum rule, K by one where the sum meets the budget within
 * rounding).  EINVAL as polar_build_frozen_set, or sum_pe_max < 0; ENOMEM;
 * ECUDA. */
int polar_build_frozen_set_device(uint32_t log2n, polar_channel ch, double param,
                                  double rate, double sum_pe_max, void *stream,
                                  polar_frozen_set **out);

/* Frozen set from the degraded-channel construction (Sec. 3's density
 * evolution made finite, after Tal & Vardy 2013): every bit-channel is
 * tracked as a symmetric channel of at most mu outputs (mu even, 2..128),
 * merged so that it stays degraded with respect to the true bit-channel;
 * its ML error probability P_e,i is therefore an upper bound that tightens
 * as mu grows (mu = 16 is within a few percent at N = 2^20).  K =
 * floor(rate * N) when rate > 0; with rate = 0, Sec. 3's rule: K is the
 * largest count whose most reliable bit-channels have sum P_e,i <=
 * sum_pe_max (an upper bound on SC's frame error rate).  The N-K largest
 * P_e,i are frozen, the lower index first on ties; polar_frozen_set_query
 * reports the sum over the information set.  Host only, double precision,
 * all host cores (about 2N mu^2 log mu operations: seconds at 2^20,
 * a minute at 2^24).  EINVAL as polar_build_frozen_set, or mu out of range,
 * or sum_pe_max < 0; ENOMEM. */
int polar_build_frozen_set_tv(uint32_t log2n, polar_channel ch, double param, int mu,
                              double rate, double sum_pe_max, polar_frozen_set **out);

/* Frozen set from a caller-given mask (bit i set = position i frozen);
 * mask_host holds max(1, N/32) words and is copied. */
int polar_frozen_set_from_mask(uint32_t log2n, const uint32_t *mask_host,
                               polar_frozen_set **out);

/* Read back N's log2, K, the mask (N/32 words, caller-owned, nullable) and
 * the sum over information bits of Z_i (BSC, a union bound on the frame
 * error rate) or P_e,i (BI-AWGN, an estimate) -- Sec. 3's FER bound.
 * Every output pointer may be NULL. */
int polar_frozen_set_query(const polar_frozen_set *fs, uint32_t *log2n,
                           uint64_t *k, uint32_t *mask_host,
                           double *sum_pe_info);

/* Make a frozen set (Sec. 3's frozen indices, as built above) resident on
 * CUDA device `device` ahead of its first SC decode (Sec. 4): its mask and
 * the node-class tables that the decoders read (the
 * subtree tables for the current "subtree_log2" and for 12, 13 and 14; for
 * "persist_log2" also the table of the levels above it).  Decodes and the
 * server otherwise upload them on first use, which on a code's first frame
 * costs host time inside that call (for the persistent server: inside
 * polar_server_submit).  Idempotent; tables stay until
 * polar_frozen_set_free.  EINVAL: NULL set or bad device; ENOMEM; ECUDA. */
int polar_frozen_set_upload(const polar_frozen_set *fs, int device);

void polar_frozen_set_free(polar_frozen_set *fs);

/* --------------------------------------------------------- channel LLRs */

/* Channel LLRs for n_total symbols (Sec. 1 and 2.2: BSC for DV-QKD, BI-AWGN
 * for CV-QKD).
 *   BSC    (y_is_bits = 1): y_dev = packed bits, L = y ? -c : c with
 *          c = ln((1-p)/p) computed in double and rounded once to float;
 *          n_total must be a multiple of 32.
 *   BIAWGN (y_is_bits = 0): y_dev = double[n_total],
 *          L = float(double(y * double(2/sigma^2))).
 * llr_dev: float[n_total].  EINVAL: NULL pointers, bad channel/parameter,
 * wrong y format for the channel. */
int polar_llr_from_channel(polar_channel ch, double param, const void *y_dev,
                           int y_is_bits, float *llr_dev, size_t n_total,
                           void *stream);

/* ------------------------------------------------------ Alice-side helpers */

/* out = in F^{(x)n} for each of nframes frames of N = 2^log2n bits (packed).
 * in_dev == out_dev is allowed.  Used by Alice to compute u = x G_N. */
int polar_encode(uint32_t log2n, int nframes, const uint32_t *in_dev,
                 uint32_t *out_dev, void *stream);

/* Syndrome-form reveal (Sec. 1): fval = (x G_N) AND mask, per frame.  This is
 * the frozen-value vector the decoders take. */
int polar_reveal(const polar_frozen_set *fs, int nframes, const uint32_t *x_dev,
                 uint32_t *fval_dev, void *stream);

/* ------------------------------------------------------------- decoding */

/* SC decoding of one frame (Sec. 4).
 *   llr_dev          float[N] channel LLRs;
 *   frozen_vals_dev  packed u with Alice's values at frozen positions (bits
 *                    at information positions are ignored);
 *   xhat_dev         packed output x_hat = u_hat G_N (Bob's estimate of x);
 *                    also used as the partial-sum store while decoding;
 *   uhat_dev         packed output u_hat, or NULL;
 *   fkind            min-sum f (bit-exact against a float32 recursive SC)
 *                    or exact f = 2 atanh(tanh(a/2) tanh(b/2)), evaluated
 *                    as sgn sgn [min + c(A+B) - c(|A-B|)] with c(d) =
 *                    ln(1 + e^-d) from the SFU exponential and logarithm,
 *                    identically at every level;
 *   prec             storage precision of the LLRs kept in device memory:
 *                    the channel LLRs as they are read and every level of
 *                    the recursion above the on-chip subtree size 2^t (FP16:
 *                    round to nearest even, saturate at +-65504; INT8: per-
 *                    frame power-of-two scale, round, saturate at +-127).
 *                    Levels below 2^t live in shared memory and registers in
 *                    float32; every f and g is computed in float32.
 * Scratch: the library grows a per-stream workspace with cudaMalloc on the
 * first call that needs more (so that call must not be inside a stream
 * capture); about N * bytes(prec) per frame. */
int polar_sc_decode(const polar_frozen_set *fs, const float *llr_dev,
                    const uint32_t *frozen_vals_dev, uint32_t *xhat_dev,
                    uint32_t *uhat_dev, polar_fkind fkind, polar_prec prec,
                    void *stream);

/* Batch of nframes frames sharing one frozen set, stored contiguously:
 * llr [nframes][N] floats, frozen_vals / xhat / uhat [nframes][N/32] words.
 * One launch sequence decodes all frames together (replayed as a CUDA graph
 * when "graphs" is on). */
int polar_sc_decode_many(const polar_frozen_set *fs, int nframes,
                         const float *llr_dev, const uint32_t *frozen_vals_dev,
                         uint32_t *xhat_dev, uint32_t *uhat_dev,
                         polar_fkind fkind, polar_prec prec, void *stream);

/* One frame of a heterogeneous batch. */
typedef struct {
    const polar_frozen_set *fs;
    const float *llr;              /* device, float[N] */
    const uint32_t *frozen_vals;   /* device, packed */
    uint32_t *xhat;                /* device, packed */
    uint32_t *uhat;                /* device, packed, or NULL */
} polar_frame_desc;

/* Frames of any lengths and frozen sets.  Consecutive frames with the same
 * frozen set whose buffers are equally strided are decoded as one batch;
 * with float32 storage the "persistent" option may instead send the whole
 * batch through polar_sc_decode_persistent. */
int polar_sc_decode_batch(int nframes, const polar_frame_desc *frames,
                          polar_fkind fkind, polar_prec prec, void *stream);

/* Frames of any lengths and frozen sets decoded by ONE persistent launch
 * (Sec. 4's SC recursion, whole frames per CTA).  The frames form a device
 * work queue, longest first; each CTA (four warps; as many per SM as shared
 * memory allows for subtrees of 2^t leaves, t = the "persist_log2" option)
 * claims the next frame and decodes it completely: the levels above t
 * stream through a per-CTA slice of the workspace, every 2^t-leaf subtree is
 * decoded in shared memory, rate-0 nodes take beta = fv F^{(x)k}.  Frames
 * never wait on one another, so a long frame overlaps many short ones.
 * Results are bit-identical to polar_sc_decode_many at the same subtree size
 * (same f and g on the same operands with the same storage rounding; min-sum
 * float32 x_hat / u_hat equal the float32 oracle).  prec: POLAR_FP32, or
 * POLAR_FP16 / POLAR_INT8 storage of the levels above t (rounded, saturated,
 * int8 with the per-frame scale of the "int8_target" option, formed by the
 * CTA itself); with reduced storage the results depend on t like those of
 * polar_sc_decode_many, which rounds the levels above its own subtree size.
 * Every llr must be 16-byte
 * aligned, frozen_vals / xhat / uhat 4-byte aligned (POLAR_EINVAL).
 * Workspace: the per-stream workspace grows (cudaMalloc) to 256 B + 64 B per
 * frame + CTAs * 4 * (2^nmax - 2^t) bytes (nmax = the longest frame), so the
 * call must not be inside a stream capture; the frame table is copied from
 * host memory with cudaMemcpyAsync before the launch returns. */
int polar_sc_decode_persistent(int nframes, const polar_frame_desc *frames,
                               polar_fkind fkind, polar_prec prec, void *stream);

/* -------------------------------------------------------------- autotuning */

/* Times the decode of this batch (contiguous as for polar_sc_decode_many)
 * under each candidate schedule -- subtree sizes t = 12, 13, 14 (float32
 * storage only: with FP16 / INT8 the rounded levels depend on t), fused and
 * unfused streamed steps, and (float32) with or without the subtree kernel
 * taking its parent's step; then, at the best t, node units of 2^s leaves
 * for s = t+1 .. t+4 (see "split_log2") with fused and unfused steps above
 * them -- then times every schedule within 4 % of the fastest again over
 * eight decodes, and keeps the fastest of that round for the batch shape
 * (device, log2 N, nframes, fkind, prec).  While the "autotune" option is 1
 * (default), later
 * decodes of that shape use it.  Synchronous on `stream`; the batch's
 * outputs are overwritten with valid decodes.  *best_fuse receives the
 * schedule flags (bit 0: fused streamed steps, bit 1: the subtree takes its
 * parent's step, bits 8..15: the node-unit level s, 0 for none).  Any of
 * best_t, best_fuse, best_ms may be NULL.  Decisions do not depend on the
 * schedule (float32); with FP16 / INT8 they depend on t only. */
int polar_autotune(const polar_frozen_set *fs, int nframes, const float *llr_dev,
                   const uint32_t *frozen_vals_dev, uint32_t *xhat_dev,
                   polar_fkind fkind, polar_prec prec, void *stream, int *best_t,
                   int *best_fuse, double *best_ms);

/* Persist / restore the tuned table as JSON (one entry per line).  load:
 * ENOTFOUND if the file is missing or holds no entry.  clear: forget all. */
int polar_tune_save(const char *path);
int polar_tune_load(const char *path);
void polar_tune_clear(void);

/* ------------------------------------------------------- verification, rate */

/* Keyed hash of each of nframes packed frames of 2^log2n bits (words_dev:
 * [nframes][max(1, N/32)] words; hash_dev: nframes uint64, device).  For
 * the verification step of Sec. 2.1: Alice and Bob hash x and x_hat with a
 * shared key and discard the blocks whose hashes differ.  h = sum_i w_i c_i
 * mod (2^61 - 1) over the frame's 32-bit words w_i, with c_i the SplitMix64
 * output number i of the key, reduced mod 2^61 - 1; with uniform
 * coefficients two different frames collide with probability 2^-61.
 * Bits of a frame shorter than a word beyond N must be zero.  EINVAL: bad
 * sizes, NULL or misaligned pointers. */
int polar_frame_hash(uint32_t log2n, int nframes, const uint32_t *words_dev, uint64_t key,
                     uint64_t *hash_dev, void *stream);

/* Secret key rate with imperfect error correction (Sec. 2.1):
 * K = alpha (1 - FER) (beta I(x:y) - S(x:E)), alpha = the decoder's output
 * rate over the data rate fed to it (at most 1), beta = R / C.  Host
 * arithmetic only. */
double polar_key_rate(double alpha, double fer, double beta, double mutual_info,
                      double eve_info);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching request server (the serving pattern around the SC
 * decoder of Sec. 4; the paper itself decodes one frame at a time).
 * Requests enter a bounded host queue and are admitted oldest first.  Two
 * modes:
 *  - slots (persistent = 0): a scheduler thread launches the oldest pending
 *    request on a free decode slot (a non-blocking CUDA stream with its own
 *    scratch) as soon as a slot is free and the scratch budget allows;
 *  - persistent (persistent = 1): one resident launch of the
 *    persistent decoder (see polar_sc_decode_persistent) whose CTAs claim
 *    frames from a ring in host-mapped memory; the scheduler publishes each
 *    admitted request's frames into the ring while the launch runs and reads
 *    per-frame completion words back, so no launch is made per request.
 *    CTAs that find nothing to do for about a millisecond leave; the
 *    scheduler relaunches when frames arrive.  Each CTA holds the scratch of
 *    the longest accepted code, 4 * 2^max_log2n bytes.
 * Either way requests that arrive while others run overlap with them on the
 * device.  The server never touches request buffers after reporting
 * completion. */
typedef struct polar_server polar_server;

typedef struct {
    int device;         /* CUDA device ordinal the server decodes on */
    int max_inflight;   /* slots: decode streams, 1..256; persistent: cap on
                           resident CTAs (frames decoded at once), 1..4096 */
    int max_queue;      /* pending requests held before submit returns EBUSY */
    size_t mem_budget;  /* bytes of decode scratch the server may hold */
    polar_fkind fkind;
    polar_prec prec;
    int threads;        /* slots: host scheduler threads launching work, 0 = 4;
                           each owns an equal share of the slots */
    int persistent;     /* 1 = persistent mode (any prec; FP16 / INT8 levels
                           are rounded above the "persist_log2" subtree size) */
    int max_log2n;      /* persistent: longest code accepted, 1..27, 0 = 22;
                           longer requests are refused at submit (EINVAL) */
} polar_server_config;

typedef struct {
    const polar_frozen_set *fs;
    int nframes;                  /* contiguous frames sharing fs, >= 1 */
    const float *llr;             /* device [nframes][N], 16-byte aligned */
    const uint32_t *frozen_vals;  /* device [nframes][N/32] */
    uint32_t *xhat;               /* device [nframes][N/32] */
    uint32_t *uhat;               /* device [nframes][N/32] or NULL */
} polar_request;

typedef struct {
    int status;         /* POLAR_OK or a negative polar_status */
    double queue_ms;    /* submit -> launch on a slot */
    double latency_ms;  /* submit -> completion observed by the scheduler */
} polar_result;

/* Start a server (EINVAL: bad config or device; ECUDA: stream creation). */
int polar_server_create(const polar_server_config *cfg, polar_server **out);

/* Queue a request; *ticket identifies it.  In persistent mode a code's first
 * request uploads its device tables inside this call (see
 * polar_frozen_set_upload, which does it ahead of time: uploads made while
 * the resident decoder runs slow it down).  EINVAL: bad request (checked on
 * the host; persistent mode also refuses codes longer than max_log2n and
 * requests of more frames than half the ring, which holds
 * max(8192, 16 * resident CTAs) frames rounded up to a power of two);
 * EBUSY: the queue holds max_queue requests (admission refused, retry
 * later).  The caller keeps every buffer alive until completion, and
 * its inputs must already be complete on the device when submit is called:
 * the server's streams do not wait on any of the caller's streams. */
int polar_server_submit(polar_server *srv, const polar_request *req, uint64_t *ticket);

/* POLAR_PENDING while the request runs; once done, its final status (OK or
 * an error: ENOMEM when its scratch alone exceeds mem_budget, ECUDA on a
 * failed launch) with *out filled, after which the ticket is forgotten.
 * ENOTFOUND for an unknown or already reported ticket. */
int polar_server_poll(polar_server *srv, uint64_t ticket, polar_result *out);

/* As poll, but blocks up to timeout_ms; ETIMEDOUT if still pending. */
int polar_server_wait(polar_server *srv, uint64_t ticket, double timeout_ms,
                      polar_result *out);

/* Withdraw a request that is still waiting in the queue (not yet launched on
 * a slot or published to the persistent ring) -- part of the serving layer
 * around Sec. 4's decoder, which the paper does not have.  Returns POLAR_OK when it was
 * withdrawn: nothing of it runs, its output buffers are never written, the
 * caller may release its buffers at once, and poll / wait then report
 * POLAR_ECANCELED for the ticket (once, like any result).  POLAR_EBUSY when
 * it has already been launched or has finished: its result arrives as usual.
 * POLAR_ENOTFOUND for an unknown or already reported ticket; POLAR_EINVAL
 * for a NULL server. */
int polar_server_cancel(polar_server *srv, uint64_t ticket);

/* Counters since creation: requests launched (slots) or published to the
 * ring (persistent), completed, refused with EBUSY, and the scratch bytes
 * the server holds.  Any pointer may be NULL. */
int polar_server_stats(polar_server *srv, uint64_t *launched, uint64_t *completed,
                       uint64_t *refused, size_t *scratch_bytes);

/* Finish queued and running requests, then release streams and scratch. */
void polar_server_destroy(polar_server *srv);

/* ------------------------------------------------- decoding, no allocation */

/* Same decisions as polar_sc_decode_many, for callers that cannot allocate
 * device memory: processes whose device memory is all owned by another
 * framework's fixed-size pool, latency-critical loops that cannot afford the
 * device synchronisation cudaMalloc and cudaFree imply, and long-running
 * services that must not meet an out-of-memory error mid-session.  The paper
 * has no counterpart; this is a deployment variant.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine and builds no
 * CUDA graph: the device copy of the frozen mask and the level scratch live
 * in one fixed, file-scope device array of polar_static_scratch_bytes()
 * bytes (16 MiB), which every GPU that loads this library holds until the
 * process exits.  The caller still passes all inputs and outputs.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     Under CUDA's lazy module loading (the default) that lookup is also when
 *     the array takes its 16 MiB of device memory, so make the first call
 *     before a memory pool claims the whole device; without room it returns
 *     POLAR_ENOMEM.
 *   - Options are read once per call: the subtree size t is the autotuned
 *     one for this batch shape when polar_autotune has an entry for it (as
 *     in polar_sc_decode_many), else the "subtree_log2" setting; "shortcuts",
 *     "fuse" and "prologue" as set.  "graphs" is ignored (launches are eager).
 *   - Capacity: the mask (N/8 bytes) and, with shortcuts on, the subtree
 *     node-class table (N/64 bytes), each rounded up to 256 bytes, plus, for
 *     INT8, nframes * 4 bytes of per-frame scales rounded up to 256, plus
 *     nframes * (N - 2^t) * bytes(prec) of levels must fit.  At t = 13 with
 *     shortcuts: up to 3 frames of 2^20 or 1 frame of 2^21 in FP32; 7 frames
 *     of 2^20 or 1 frame of 2^22 in FP16; 15 frames of 2^20 or 3 frames of
 *     2^22 in INT8.  Larger requests return POLAR_EINVAL before any launch,
 *     with the sizes in polar_last_error_string().
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the mask and class table are rewritten each call, the INT8
 *     scales are written before they are read, and so is every scratch
 *     level.  Calls whose work overlaps on the GPU (other streams, other
 *     host threads) race on the array: serialise them. */
int polar_sc_decode_many_noalloc(const polar_frozen_set *fs, int nframes,
                                 const float *llr_dev, const uint32_t *frozen_vals_dev,
                                 uint32_t *xhat_dev, uint32_t *uhat_dev,
                                 polar_fkind fkind, polar_prec prec, void *stream);

/* Size in bytes of the static array behind polar_sc_decode_many_noalloc. */
size_t polar_static_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* POLAR_GB300_H */

/*
 * twofold.h -- C ABI of the GB300 twofold library.
 *
 * Twofold fast arithmetic (E. Latkin, "Twofold fast arithmetic",
 * arXiv:1401.6235): a value z is carried as z ~ z0 + z1 where z0 is bit for
 * bit the plain IEEE binary64 result of the same computation and z1
 * estimates its error dz0 = z - z0 (Algorithms, "Methodic").  Every entry
 * point below returns, per result, z0, z1 and a panic flag byte.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 *  - Arrays are structure-of-arrays: a twofold array is a pair of binary64
 *    arrays `hi` (z0) and `lo` (z1).  `lo == NULL` marks a "dotted" input: a
 *    plain binary64 value with no tail, which selects the paper's ".1"
 *    algorithms (see twofold_ew for the exact rule).
 *  - Unless stated otherwise, data pointers are DEVICE pointers owned by the
 *    caller (for example torch tensors); the library does not allocate,
 *    free or synchronise data memory.  The exceptions are the request server
 *    below, which owns a device arena and a scheduler thread;
 *    twofold_dot_noalloc, whose partials live in a static device array; and
 *    the run-time specialised elementwise kernels, which are compiled and
 *    loaded once per program (code memory, see twofold_ew_jit).  Every call
 *    is asynchronous on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream).
 *  - Pinned host memory that the device maps at the same address (memory
 *    from cudaHostAlloc / cudaMallocHost under unified addressing;
 *    twofold_host_mapped tells) may stand in for device memory in the data
 *    arrays of twofold_ew, plain_ew, twofold_ew_f32, plain_ew_f32, of the
 *    single twofold_sum / twofold_dot and of twofold_horner(_batched)
 *    (points and results; coefficients and workspaces stay device memory): the kernels then read their inputs and
 *    write their results across the host link themselves.  The arithmetic
 *    is the same device code with the same bits.
 *  - Device data pointers must be 8-byte aligned (flags: any alignment).
 *    Lengths are element counts; n == 0 is valid, and then data pointers
 *    that would not be read or written may be NULL.
 *  - Results are deterministic and independent of launch configuration:
 *    z0, z1 and flags are bit-identical to the CPU oracle of the same
 *    operation order (NaN payloads excepted).
 *  - NaN and Inf are not errors (Algorithms, "Methodic": no special-case
 *    processing); they propagate through the basic operations and raise
 *    TF_FLAG_NONFINITE.
 *  - Return value: TF_OK or a negative tf_status.  Argument errors are
 *    detected before any launch (nothing is written); TF_ECUDA reports a
 *    launch error (cudaGetLastError) and leaves outputs undefined.
 *  - Compiled with -fmad=false and explicit round-to-nearest intrinsics:
 *    no multiply-add is contracted, so z0 is the plain IEEE result.
 */
#ifndef TWOFOLD_H
#define TWOFOLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- types */

/* A twofold input array: hi = z0 values; lo = z1 tails, or NULL (dotted). */
typedef struct {
    const double *hi;
    const double *lo;
} tf_in;

/* A twofold output array.  hi and lo are required (n doubles each, or one
 * per job for reductions); flags is optional (NULL: not written). */
typedef struct {
    double *hi;
    double *lo;
    uint8_t *flags;
} tf_out;

/* Panic flag (Motivation: the "twofold daemon" that signals when z1 gets
 * large compared with z0; the paper fixes no threshold):
 *   TF_PANIC_REL: PANIC when |z1| > panic_tau * |z0|   (default tau = 2^-40)
 *   TF_PANIC_ULP: PANIC when |z1| > panic_ulps * ulp(z0),
 *                 ulp(v) = 2^(max(e,-1022)-52) for v = 1.f * 2^e, ulp(0) = 2^-1074
 * Both products are single round-to-nearest multiplications.  NaN compares
 * false, so a NaN z1 never raises PANIC; NONFINITE covers it.
 * panic_mode | TF_PANIC_STICKY (elementwise programs): the flag of a result
 * ORs the flags of every instruction's result of its program, so a loss of
 * accuracy anywhere in a chain stays visible at its end. */
enum { TF_PANIC_REL = 0, TF_PANIC_ULP = 1, TF_PANIC_STICKY = 4 };
enum { TF_FLAG_PANIC = 1, TF_FLAG_NONFINITE = 2 };

typedef struct {
    int32_t panic_mode;   /* TF_PANIC_REL or TF_PANIC_ULP, | TF_PANIC_STICKY   */
    int32_t leaf;         /* leaf length L of sum/dot (>= 1); default 256      */
    double  panic_tau;    /* REL threshold >= 0, default 0x1p-40               */
    double  panic_ulps;   /* ULP threshold m >= 0, default 4096                */
} tf_params;              /* a NULL tf_params* means all defaults              */

typedef enum {
    TF_OK = 0,
    TF_EINVAL = -1,        /* bad argument (NULL, misaligned, n < 0, bad program, ...) */
    TF_ENOSPC = -2,        /* workspace too small                                     */
    TF_ECUDA = -3,         /* CUDA launch / runtime error                             */
    TF_ETIMEOUT = -4,      /* a bounded device-side wait gave up                      */
    TF_EUNSUPPORTED = -5   /* valid request outside the library's limits             */
} tf_status;

/* Human-readable text of a status code (static storage). */
const char *twofold_strerror(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int twofold_version(void);

/* 1 when `ptr` is host memory that the current device accesses at the same
 * address (page-locked and mapped, see the conventions above), else 0 (also
 * for device memory, ordinary pageable memory, NULL, or when no device is
 * present).  No paper counterpart: a query for the host-buffer form of the
 * elementwise entry points.  Never fails; clears the CUDA error it may raise. */
int twofold_host_mapped(const void *ptr);

/* --------------------------------------------------- elementwise programs
 *
 * twofold_ew -- evaluate a straight-line program over n twofold elements.
 *
 * Operations (Algorithms section):
 *   TF_ADD  Add/subtract, Algorithm ATF 1  (ATF 1.1 when b is dotted)
 *   TF_SUB  Add/subtract, Algorithm STF 1  (STF 1.1 when b is dotted)
 *   TF_MUL  Multiply,     Algorithm MTF 1  (MTF 1.1 when b is dotted)
 *   TF_DIV  Divide,       Algorithm DTF 1  (DTF 1.1 when b is dotted)
 *   TF_SQRT Root,         Algorithm RTF 1  (RPF 1.1 when a is dotted)
 * with err() of sums and differences from Algorithms 1.2 / 2.2, products
 * from Algorithm 3, remainders from Algorithms 4 and 5 (Background).
 * Operand kinds: both twofold -> the general algorithm; a twofold, b dotted
 * -> the ".1" algorithm; a dotted, b twofold -> the general algorithm with
 * a's tail = +0; both dotted -> the exact transform (Two-Sum, Two-Diff,
 * Two-Product) or DTF 1.1.1.  Only inputs can be dotted; every
 * intermediate is a general twofold.
 *
 * Coupled ("p", Dekker emulation) operations, the paper's p-prefixed
 * functions (Dekker arithmetic section, Algorithms, Applications): the
 * algorithm for non-overlapping operands, then the result renormalised with
 * Fast Two-Sum (Algorithm 1.1, its three operations as printed):
 *   TF_PADD  ATF 1 (ATF 1.1)      TF_PSUB  STF 1 (STF 1.1)
 *   TF_PMUL  MPF 1 (MTF 1.1)      TF_PDIV  DPF 1 (DTF 1.1)
 *   TF_PSQRT RPF 1
 * (in brackets: b dotted).  With every operand dotted the exact transform,
 * DTF 1.1.1 or RPF 1.1 is returned unrenormalised (already coupled).  Their
 * z0 is the renormalised head, not the plain result; plain_ew evaluates
 * them as the basic operation.
 *
 * prog    HOST array of nprog instructions, 4 int32 each: {op, dst, a, b}.
 *         Registers 0..nin-1 are the inputs (read only); registers
 *         nin..TF_EW_MAX_REGS-1 are temporaries.  a and b must name an input
 *         or a temporary written by an earlier instruction; b is ignored
 *         for TF_SQRT and TF_PSQRT.  The result is the last instruction's dst.
 * nprog   1..TF_EW_MAX_PROG.
 * in      HOST array of nin tf_in descriptors (device data pointers).
 * nin     1..TF_EW_MAX_INPUTS.
 * n       elements (>= 0); every input and output array holds n values.
 * out     z0, z1 (n doubles each) and optional flags (n bytes).
 * p       panic parameters (NULL: defaults).
 * Errors: TF_EINVAL for a malformed program or bad pointers.
 */
enum { TF_ADD = 1, TF_SUB = 2, TF_MUL = 3, TF_DIV = 4, TF_SQRT = 5,
       TF_PADD = 6, TF_PSUB = 7, TF_PMUL = 8, TF_PDIV = 9, TF_PSQRT = 10 };
enum { TF_EW_MAX_PROG = 32, TF_EW_MAX_INPUTS = 12, TF_EW_MAX_REGS = 32 };

int twofold_ew(const int32_t *prog, int32_t nprog, const tf_in *in, int32_t nin,
               int64_t n, tf_out out, const tf_params *p, void *stream);

/* Runtime specialisation of elementwise programs: for n >= 2^20 (automatic
 * mode) twofold_ew and twofold_ew_f32 run a straight-line kernel of the
 * program, compiled once per distinct program (and operand kinds and flag
 * mode) at its first such call by the runtime compiler for this GPU from the
 * library's own device code, and cached for the process; its results are the
 * generic kernels' bits.  A program that cannot be compiled runs on the
 * generic kernels.  twofold_ew_jit sets the mode (0 off, 1 automatic, 2 at
 * every size; -1 only queries), returns the previous one (the initial mode is
 * $TWOFOLD_JIT when set, else 1), and reports how many kernels were built
 * and failed so far (either pointer may be NULL).  No paper counterpart. */
int twofold_ew_jit(int32_t mode, int64_t *built, int64_t *failed);

/* Plain binary64 twin of twofold_ew: the same program on the hi arrays
 * only (in: HOST array of nin device pointers), out[i] = the plain result
 * (a coupled op evaluates as its basic op).  It equals twofold_ew's z0 bit
 * for bit for programs without coupled ops. */
int plain_ew(const int32_t *prog, int32_t nprog, const double *const *in, int32_t nin,
             int64_t n, double *out, void *stream);

/* Arithmetic of the plain binary64 twins, for measuring the twofold kernels
 * against the fastest plain twin as well as the usual one:
 *   TF_PLAIN_NATIVE  (0, initial): CUDA's operations, what a plain binary64
 *                    kernel compiles to (__ddiv_rn, __dsqrt_rn, __dmul_rn);
 *   TF_PLAIN_INTEGER (1): the library's integer-pipe routines where they are
 *                    faster on this GPU, the ones the twofold kernels use:
 *                    the division and square root of plain_ew (Algorithms 4
 *                    and 5's quotient and root) and the multiplication of
 *                    plain_horner(_batched).  All are correctly rounded: the
 *                    results are the same bits.
 * mode -1 only queries.  Returns the previous mode, or TF_EINVAL for any
 * other mode.  The setting is process-wide and read when a plain call is
 * made (set it while no other thread makes one).  The plain sum and dot
 * keep the native operations in both modes (an integer multiplication made
 * the plain dot slower), as do the binary32 twins.  No paper counterpart. */
#define TF_PLAIN_NATIVE 0
#define TF_PLAIN_INTEGER 1
int plain_arith(int32_t mode);

/* ------------------------------------------- binary32 elementwise programs
 *
 * The same programs, operations, operand kinds and flags over binary32
 * twofolds (the paper's algorithms are generic over the number type; its
 * logs print float rows).  Every operation is a round-to-nearest binary32
 * operation with subnormals kept.  Flags: tau and ulps of `p` are rounded to
 * binary32; with p == NULL, tau = 2^-18 (the share of binary32's 24-bit
 * significand that 2^-40 is of binary64's 53) and ulps = 4096.  Pointers
 * are 4-byte aligned device (or mapped host) pointers. */
typedef struct {
    const float *hi;
    const float *lo;
} tf_in_f32;

typedef struct {
    float *hi;
    float *lo;
    uint8_t *flags;
} tf_out_f32;

int twofold_ew_f32(const int32_t *prog, int32_t nprog, const tf_in_f32 *in, int32_t nin,
                   int64_t n, tf_out_f32 out, const tf_params *p, void *stream);
int plain_ew_f32(const int32_t *prog, int32_t nprog, const float *const *in, int32_t nin,
                 int64_t n, float *out, void *stream);

/* ------------------------------------------------------ sum and dot
 *
 * Reduction order (the paper fixes none; "2x" section: a twofold
 * accumulator summing plain values is strict per step, Algorithm ATF 1.1):
 *   - leaves are consecutive blocks of L = p->leaf elements (the last may
 *     be short); each leaf runs acc = (+0, +0), acc = ATF1(acc, term_i)
 *     from left to right, where term_i is x_i (ATF 1.1 when x is dotted)
 *     for a sum, or the twofold product of x_i and y_i for a dot (Two-
 *     Product when both are dotted, MTF 1 when both are twofold, MTF 1.1
 *     when only y is dotted, MTF 1 with x1 = +0 when only x is dotted);
 *   - the leaf results are combined by a bottom-up pairwise tree: node i
 *     of level j+1 = ATF1(node 2i, node 2i+1) of level j, an odd last node
 *     is carried up unchanged; the root is the result (n = 0: (+0, +0)).
 * Node i of level j covers leaves [i 2^j, min((i+1) 2^j, m)), so any
 * aligned 2^k-leaf block is a subtree: the GPU reduces blocks in parallel
 * and combines their partials in the same order.
 *
 * out1    one result: out1.hi[0], out1.lo[0], out1.flags[0] (optional).
 * ws      DEVICE workspace of ws_bytes >= twofold_workspace_bytes(...);
 *         its contents on entry are irrelevant; it is scratch until the
 *         stream reaches the end of the call.
 * Errors: TF_ENOSPC if ws_bytes is too small.
 */
enum { TF_KIND_SUM = 1, TF_KIND_DOT = 2 };

size_t twofold_workspace_bytes(int32_t kind, int64_t n_total, int32_t njobs,
                               const tf_params *p);

int twofold_sum(tf_in x, int64_t n, tf_out out1, const tf_params *p,
                void *ws, size_t ws_bytes, void *stream);
int twofold_dot(tf_in x, tf_in y, int64_t n, tf_out out1, const tf_params *p,
                void *ws, size_t ws_bytes, void *stream);

/* Batched (one launch for all jobs): job j reduces elements
 * [offs[j], offs[j+1]) of x (and y) and writes out.hi[j], out.lo[j],
 * out.flags[j].  offs is a HOST array of njobs+1 non-decreasing int64 with
 * offs[0] >= 0; the job table derived from it is uploaded into ws with
 * cudaMemcpyAsync (the call returns once the host array may be reused).
 * Jobs of any lengths may be mixed; each result equals the single-job call. */
int twofold_sum_batched(tf_in x, const int64_t *offs, int32_t njobs, tf_out out,
                        const tf_params *p, void *ws, size_t ws_bytes, void *stream);
int twofold_dot_batched(tf_in x, tf_in y, const int64_t *offs, int32_t njobs, tf_out out,
                        const tf_params *p, void *ws, size_t ws_bytes, void *stream);

/* Plain binary64 twins: the same leaves and tree with s = +0; s = s (+) x_i
 * (sum) or s = s (+) (x_i (*) y_i) (dot, separate multiply and add).  They
 * equal the twofold z0 bit for bit.  out: one double per job (device). */
int plain_sum(const double *x, int64_t n, double *out1, const tf_params *p,
              void *ws, size_t ws_bytes, void *stream);
int plain_dot(const double *x, const double *y, int64_t n, double *out1, const tf_params *p,
              void *ws, size_t ws_bytes, void *stream);
int plain_dot_batched(const double *x, const double *y, const int64_t *offs, int32_t njobs,
                      double *out, const tf_params *p, void *ws, size_t ws_bytes, void *stream);

/* Twofold sum and dot over binary32 twofolds (the paper's float basis), in
 * the same blocked pairwise order as twofold_sum / twofold_dot (leaves of
 * p->leaf elements, ATF1 / ATF1.1 accumulation, products by the operand
 * kinds, the pairwise tree with the odd node carried); one result, its
 * panic flag from p (binary32 defaults: REL with tau = 2^-18).  x.lo / y.lo
 * NULL: dotted input.  Pointers are device pointers aligned to 4 bytes.
 * ws: at least twofold_workspace_bytes(kind, n, 1, p) bytes (8-byte
 * aligned).  n == 0 gives (+0, +0) and flag 0.  The plain twins compute
 * the same order in plain binary32 (s + x_i, s + x_i * y_i). */
int twofold_sum_f32(tf_in_f32 x, int64_t n, tf_out_f32 out1, const tf_params *p, void *ws, size_t ws_bytes,
                    void *stream);
int twofold_dot_f32(tf_in_f32 x, tf_in_f32 y, int64_t n, tf_out_f32 out1, const tf_params *p, void *ws,
                    size_t ws_bytes, void *stream);
int plain_sum_f32(const float *x, int64_t n, float *out1, const tf_params *p, void *ws, size_t ws_bytes,
                  void *stream);
int plain_dot_f32(const float *x, const float *y, int64_t n, float *out1, const tf_params *p, void *ws,
                  size_t ws_bytes, void *stream);

/* The upper levels of the reduction order over m partial results (z0[i],
 * z1[i] device arrays): the pairwise tree with the odd node carried, then
 * the panic flag, as a sum or dot ends.  When the partials are the results
 * of consecutive aligned blocks of 2^k leaves of one sum or dot (for
 * example one block per GPU of a sharded reduction), the result is the
 * whole reduction's, bit for bit.  m == 0 gives (+0, +0).  ws_bytes >=
 * 2 * 256-rounded 8m bytes (the partials are copied there first; the inputs
 * are not modified).  No paper counterpart: the multi-GPU split's combine. */
int twofold_combine(const double *z0, const double *z1, int64_t m, tf_out out1, const tf_params *p,
                    void *ws, size_t ws_bytes, void *stream);

/* Dot product that allocates nothing and takes no workspace (the paper has
 * no counterpart: this is an interface for callers that cannot provide
 * device memory at the call, e.g. code that must not touch the allocator
 * once running or that has no spare buffer to lend).  Same arguments,
 * order and results as twofold_dot without ws.  Its scratch is a static
 * 512 KiB device array of the library (up to 32768 reduction blocks, about
 * 2^31 elements at the default leaf of 256), held on every GPU that loads
 * the library until exit; larger requests return TF_EUNSUPPORTED before any
 * launch.  The first call on a device looks up the array's address with
 * cudaGetSymbolAddress (make it before any stream capture) and keeps it for
 * the rest of the process: it belongs to the device's primary context, so
 * after cudaDeviceReset, or under a driver context other than the primary
 * one, this entry point must not be called on that device.  All calls
 * share the array: calls that overlap on the GPU race; calls ordered on one
 * stream do not. */
int twofold_dot_noalloc(tf_in x, tf_in y, int64_t n, tf_out out1, const tf_params *p, void *stream);

/* The number of bounded device-side waits that ran out on the current
 * device since the library was loaded (no paper counterpart: a diagnostic).
 * The latency schedule of twofold_sum / twofold_dot (few leaves) runs each
 * block of leaves on a pair of CTAs on two SMs, one handing chunks of its
 * results to the other; the receiving CTA waits for each chunk a bounded
 * number of polls, and if a wait runs out the block's result is NaN and
 * this count grows.  Synchronous: it waits for the device's pending work
 * in the legacy default stream.  TF_ECUDA if the count cannot be read. */
int twofold_wait_timeouts(uint64_t *count);

/* Failure injection for testing the bounded waits above (no paper
 * counterpart; no device fault is involved): from this call on, the latency
 * schedule's producer CTAs do not send the tails of chunk `chunk` of each
 * leaf (chunks count from 0), and the receiving CTAs give up waiting after
 * 2^12 polls instead of 2^24; each affected block's result is NaN and
 * twofold_wait_timeouts grows by one per block.  chunk = -1 turns injection
 * off.  Process-wide, read when a sum or dot is launched.  Returns the
 * previous setting, or TF_EINVAL for a chunk outside -1 .. 11. */
int twofold_inject_pair_drop(int32_t chunk);

/* -------------------------------------------------------------- Horner
 *
 * p(x) = a_0 + a_1 x + ... + a_k x^k with dotted coefficients (ascending)
 * and dotted points: s = (a_k, +0); for i = k-1 .. 0:
 *     s = ATF 1.1( MTF 1.1(s, x), a_i )
 * (Multiply: MTF 1.1; Add/subtract: ATF 1.1; the composition is not in the
 * paper).  One result per point.
 *
 * coef    DEVICE array of k+1 doubles, a_0 first.  0 <= k <= TF_HORNER_MAX_K.
 * x       DEVICE array of n points; out: n results.
 */
enum { TF_HORNER_MAX_K = 1024 };

int twofold_horner(const double *coef, int32_t k, const double *x, int64_t n, tf_out out,
                   const tf_params *p, void *stream);

/* Batched: job j evaluates the degree-ks[j] polynomial with coefficients
 * coefs[coef_offs[j] .. coef_offs[j] + ks[j]] at points
 * x[x_offs[j] .. x_offs[j+1]), writing out at the same indices.
 * coefs and x are DEVICE arrays; coef_offs, ks (njobs each) and x_offs
 * (njobs+1, non-decreasing, x_offs[0] >= 0) are HOST arrays, uploaded into
 * ws (ws_bytes >= twofold_horner_workspace_bytes(njobs)). */
size_t twofold_horner_workspace_bytes(int32_t njobs);
int twofold_horner_batched(const double *coefs, const int32_t *coef_offs, const int32_t *ks,
                           int32_t njobs, const double *x, const int64_t *x_offs, tf_out out,
                           const tf_params *p, void *ws, size_t ws_bytes, void *stream);

/* Plain twins: s = a_k; s = (s (*) x) (+) a_i, no FMA. */
int plain_horner(const double *coef, int32_t k, const double *x, int64_t n, double *out,
                 void *stream);
int plain_horner_batched(const double *coefs, const int32_t *coef_offs, const int32_t *ks,
                         int32_t njobs, const double *x, const int64_t *x_offs, double *out,
                         void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------- mixed persistent batches
 *
 * Sum, dot and Horner jobs of any number and sizes in ONE persistent launch.
 * No paper counterpart (a GPU interface): every job's result is the result
 * of its single-job entry point (twofold_sum, twofold_dot, twofold_horner
 * with the same tf_params), bit for bit, whatever the mix and the config.
 *
 * Work items are an aligned block of B = cfg->leaves_per_item leaves of a
 * sum/dot job, or a range of cfg->points_per_item points of a Horner job.
 * A job of more than B leaves is split into several items; since an aligned
 * block of 2^k leaves is a subtree of the blocked pairwise order (see
 * twofold_sum), the CTA that completes the job's last item combines the
 * item partials with the same tree.  Resident CTAs take items largest first
 * from an atomic counter; no CTA ever waits for another.
 *
 * twofold_batch_prepare validates the jobs (as the single-job calls do),
 * builds the job and item tables and zeroes the counters in `ws`
 * (ws_bytes >= twofold_batch_workspace_bytes(...), 256-byte aligned) with
 * stream-ordered copies from host memory (it may wait for earlier work on
 * `stream`), and fills `plan`.  twofold_batch_launch starts the persistent
 * kernel of a prepared plan: it does no host work besides the launch, so it
 * may be captured into a CUDA graph and replayed; the kernel leaves the
 * counters zeroed for the next launch.  Launches of one plan must not
 * overlap (one stream), and the plan's workspace and the jobs' buffers must
 * stay valid.  twofold_batch = prepare + launch.
 *
 * Jobs: tf_job.kind TF_JOB_SUM / TF_JOB_DOT: x (and y) as in twofold_sum /
 * twofold_dot, one result at out.hi[0], out.lo[0] (out.flags[0] if
 * non-NULL); n == 0 gives (+0, +0).  TF_JOB_HORNER: degree k in
 * [0, TF_HORNER_MAX_K], coefs (k+1 ascending, device), points x.hi (x.lo
 * NULL), n results in out.  All pointers device pointers.
 * Config (NULL: defaults): leaves_per_item a power of two in [1, threads]
 * (256), points_per_item >= 1 (16384), threads 128 / 256 / 512 (256),
 * ctas_per_sm >= 0 (0: by occupancy).  Errors: TF_EINVAL (bad job, config
 * or plan), TF_ENOSPC (workspace too small or not 256-byte aligned),
 * TF_EUNSUPPORTED (more than 2^31 - 1
 * items), TF_ECUDA. */
enum { TF_JOB_SUM = 1, TF_JOB_DOT = 2, TF_JOB_HORNER = 3 };

typedef struct {
    int32_t kind;          /* TF_JOB_SUM, TF_JOB_DOT or TF_JOB_HORNER            */
    int32_t k;             /* Horner degree                                      */
    int64_t n;             /* elements (sum, dot) or points (Horner), >= 0       */
    tf_in x;               /* operand / Horner points in x.hi                    */
    tf_in y;               /* dot: second operand                                */
    const double *coefs;   /* Horner coefficients                                */
    tf_out out;            /* results                                            */
} tf_job;

typedef struct {
    int32_t leaves_per_item;
    int32_t points_per_item;
    int32_t threads;
    int32_t ctas_per_sm;
} tf_batch_config;

typedef struct { int64_t opaque[16]; } tf_batch_plan;   /* filled by twofold_batch_prepare */

size_t twofold_batch_workspace_bytes(const tf_job *jobs, int32_t njobs, const tf_params *p,
                                     const tf_batch_config *cfg);   /* 0 for an invalid list */
int twofold_batch_prepare(const tf_job *jobs, int32_t njobs, const tf_params *p,
                          const tf_batch_config *cfg, void *ws, size_t ws_bytes, tf_batch_plan *plan,
                          void *stream);
int twofold_batch_launch(const tf_batch_plan *plan, void *stream);
int twofold_batch(const tf_job *jobs, int32_t njobs, const tf_params *p, const tf_batch_config *cfg,
                  void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------ serving loop
 *
 * A request server (no paper counterpart: a serving interface over the
 * entry points above).  twofold_server_create reserves a device arena of
 * mem_cap_bytes (the only entry point that allocates device memory) and
 * starts one scheduler thread.  Requests carry HOST buffers; they wait in
 * FIFO order, and whenever memory and a stream are free the scheduler admits
 * the longest prefix of the queue that fits the arena (inputs, outputs and
 * the batch workspace), up to max_batch_jobs requests and a quarter of
 * mem_cap_bytes of request buffers (a larger single request is admitted
 * alone), copies the inputs in,
 * runs the sum / dot / Horner requests as one mixed persistent batch
 * (twofold_batch, with `cfg`) and the elementwise requests as twofold_ew
 * launches, copies the results out and releases the memory when the batch's
 * event fires.  Up to three batches are in flight on a pool of streams, so
 * requests that arrive while others run are admitted as memory frees up and
 * their copies and kernels overlap.  A request's results are those of the
 * single-job entry point on the same inputs (the same bits), alone or in any
 * mix.  A request larger than the whole arena fails with TF_ENOSPC.
 *
 * Requests (tf_request): kind TF_JOB_SUM (in[0] = x, in[1] = x tails or
 * NULL), TF_JOB_DOT (in[0..3] = x, x tails, y, y tails; tails may be NULL),
 * TF_JOB_HORNER (in[0] = points, coefs = k+1 coefficients), TF_JOB_EW
 * (program prog/nprog as for twofold_ew over nin <= 4 twofold inputs,
 * in[2i] = hi, in[2i+1] = lo or NULL; the program is copied at submit).
 * Outputs: out_hi, out_lo (1 result for sum/dot, n for Horner and
 * elementwise), out_flags optional.  All in/out pointers are HOST pointers
 * that must stay valid until twofold_server_wait returns for the ticket;
 * page-locked outputs let the copies run asynchronously (pageable ones make
 * the scheduler wait for them).  Every ticket must be waited for once.
 *
 * twofold_server_wait blocks until the request is done (timeout_ms < 0:
 * without limit) and returns its status (TF_ETIMEOUT when the time ran out;
 * the ticket stays valid), filling `info` with host clock stamps
 * (steady clock, ns) of submission, admission and completion and the size
 * of the batch the request ran in.  twofold_server_destroy finishes every
 * pending request, stops the thread and frees the arena. */
enum { TF_JOB_EW = 4 };

typedef struct tf_server tf_server;

typedef struct {
    int32_t kind;
    int32_t k;                 /* Horner degree                              */
    int64_t n;                 /* elements / points                          */
    const double *in[8];       /* host inputs, see above                     */
    const double *coefs;       /* Horner coefficients (host)                 */
    const int32_t *prog;       /* elementwise program (host, nprog rows of 4) */
    int32_t nprog;
    int32_t nin;               /* elementwise twofold inputs (1..4)          */
    double *out_hi;            /* host outputs                               */
    double *out_lo;
    uint8_t *out_flags;
} tf_request;

typedef struct {
    int64_t submitted_ns, admitted_ns, done_ns;
    int32_t status;            /* TF_OK or a negative tf_status              */
    int32_t batch_jobs;        /* requests in the batch it ran in            */
} tf_request_info;

typedef struct {
    int64_t completed, failed, batches, batched_jobs;
    int64_t arena_bytes, peak_bytes, pending;
    int32_t max_inflight, inflight;
} tf_server_stats;

int twofold_server_create(size_t mem_cap_bytes, int32_t max_batch_jobs, const tf_params *p,
                          const tf_batch_config *cfg, tf_server **out);
int twofold_server_submit(tf_server *s, const tf_request *r, uint64_t *ticket);
int twofold_server_wait(tf_server *s, uint64_t ticket, int32_t timeout_ms, tf_request_info *info);
int twofold_server_stats(tf_server *s, tf_server_stats *out);
int twofold_server_destroy(tf_server *s);

/* Host-side fault injection, for testing what callers of the server see
 * when a batch fails (no paper counterpart; no device fault is involved):
 * from this call on, every `every`-th batch the scheduler starts is failed
 * before any of its copies or launches, as if one of its CUDA calls had
 * returned an error.  Its requests complete with TF_ECUDA (counted in the
 * stats' `failed`), its memory is released, and the server goes on with the
 * following batches.  every = 0 turns injection off; every < 0 (or s NULL)
 * is TF_EINVAL. */
int twofold_server_inject_failures(tf_server *s, int32_t every);

/* ------------------------------------------------------ pipe-rate probes
 *
 * Measurement only (no paper counterpart): the binary64 kernels above are
 * bound by the SM's FP64 pipe and integer pipes, so their roofline is the
 * rate at which an SM retires each instruction kind.  One launch of
 * `blocks` CTAs of `threads` threads (a multiple of 32, at most 1024) runs,
 * per thread, `iters` x 128 instructions of kind `op` over 8 independent
 * register chains:
 *   TF_PROBE_DADD / DMUL / DFMA   binary64 add / multiply / fused multiply-add
 *   TF_PROBE_FFMA                 binary32 fused multiply-add (the FMA pipe;
 *                                 at full rate it shows the issue limit)
 *   TF_PROBE_IMAD                 32-bit integer multiply-add
 *   TF_PROBE_SHF                  32-bit funnel shift (the integer ALU pipe)
 *   TF_PROBE_MULHI64              high half of a 64 x 64-bit product
 *   TF_PROBE_MUFU                 binary32 reciprocal square-root
 *                                 approximation (the special-function unit
 *                                 that seeds the integer division and root)
 *   TF_PROBE_I2F                  32-bit unsigned to binary32 conversion
 * op | TF_PROBE_LATENCY (DADD, DMUL, DFMA, IMAD only) runs the same count as
 * one dependent chain per thread: with one warp per SM, 32 / (lane ops per
 * SM clock) is the latency of one instruction in SM clocks.
 * TF_PROBE_LATENCY | TF_PROBE_CHAIN_LDS runs a short reduction's critical
 * loop: per element one 16-byte shared-memory load and two dependent
 * binary64 adds, iters x 256 elements per thread (not x 128 instructions):
 * with one warp per SM, 32 x 2 / (lane ops per SM clock) is the clocks one
 * element takes.  TF_PROBE_LATENCY | TF_PROBE_CHAIN_AHEAD runs the same loop
 * with its loads and adds in a fixed order, each 8 elements' loads issued
 * right after the first add of the 8 before.
 * CTA b writes rec[4b .. 4b+3] (device int64 array of 4 * blocks, 8-byte
 * aligned): its SM id, its start and end SM clock (clock64), and a digest
 * of its chains.  Lane operations per SM clock on SM s = (threads x iters x
 * 128 x the CTAs that ran on s) / (last end - first start on s).  Size the
 * grid so that all CTAs are resident at once.  Asynchronous on `stream`;
 * TF_EINVAL for an unknown op or bad sizes, TF_ECUDA for a launch error. */
#define TF_PROBE_DADD 0
#define TF_PROBE_DMUL 1
#define TF_PROBE_DFMA 2
#define TF_PROBE_FFMA 3
#define TF_PROBE_IMAD 4
#define TF_PROBE_SHF 5
#define TF_PROBE_MULHI64 6
#define TF_PROBE_MUFU 7
#define TF_PROBE_I2F 8
#define TF_PROBE_CHAIN_LDS 9
#define TF_PROBE_CHAIN_AHEAD 10
#define TF_PROBE_LATENCY 0x100
int twofold_pipe_probe(int32_t op, int64_t iters, int32_t blocks, int32_t threads, int64_t *rec, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TWOFOLD_H */

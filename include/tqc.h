/*
 * tqc.h -- C ABI of the GB300 cut-network reconstruction library (libtqc.so).
 *
 * What the library computes (Eq. reconstruction, §II-A, and its tensor-network
 * form, §III-B): given the m subcircuit output tensors of a cut circuit, each
 * indexed by its output bits (dimension 2) and its cut edges (dimension 4,
 * basis order I, X, Y, Z), the uncut circuit's output probabilities
 *
 *     P(x) = 2^{-|E|} sum_{e in {I,X,Y,Z}^{|E|}} prod_j T_j[e|E_j][x|out_j]
 *
 * for every state x of a requested bin, by a sequence of m-1 pairwise
 * contractions (§III-B, Fig. subcircuit_contraction) in an order chosen by a
 * planner (§III-E-1), with index slicing when tensors exceed a memory budget
 * (§III-E-2).  The factor 1/2 per cut is applied once, exactly, at the end.
 *
 * Conventions
 *   - Qubit q of a state is bit q of its index (little-endian); n_qubits <= 128.
 *   - A bin fixes some qubits to given bits and leaves F qubits free.  Output
 *     entry i (0 <= i < 2^F) is the state whose i-th free qubit (free qubits in
 *     ascending order) carries bit i of the index; F <= 40.
 *   - All errors are returned as tqc_status; no C++ exception crosses the ABI.
 *     tqc_last_error() returns a thread-local message describing the last
 *     failure on the calling thread (naming the offending subcircuit or cut for
 *     validation errors).
 *   - Device work is stream-ordered on the caller's stream.  After the first
 *     tqc_contract on a plan (which allocates the plan's workspace), further
 *     calls with z_out == NULL neither allocate nor synchronise.
 *   - Handles are not thread-safe: one thread uses a plan at a time.
 *   - A plan's workspace (and its K-split partials) serve every call on it:
 *     calls on the same plan must not overlap on the GPU (issue them on one
 *     stream, or order the streams with events).  Different plans may run
 *     concurrently.
 */
#ifndef TQC_H_
#define TQC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TQC_API __attribute__((visibility("default")))
#else
#define TQC_API
#endif

typedef struct tqc_net *tqc_net_t;
typedef struct tqc_plan *tqc_plan_t;

typedef enum {
    TQC_OK = 0,
    TQC_ERR_INVALID = 1,      /* bad argument, label or layout */
    TQC_ERR_OOM = 2,          /* device or host allocation failed, or budget too small */
    TQC_ERR_CUDA = 3,         /* a CUDA call failed (message holds cudaGetErrorString) */
    TQC_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    TQC_ERR_UNSUPPORTED = 5   /* valid request outside what the library supports */
} tqc_status;

/* element types of tensors and outputs */
enum { TQC_F64 = 0, TQC_F32 = 1 };

/* arithmetic form of the pairwise contractions */
enum {
    TQC_PREC_FP32 = 0,   /* plain form: every step on CUDA cores in FP32 */
    TQC_PREC_TF32 = 1,   /* dense steps on tcgen05 tensor cores, TF32 inputs, FP32 accumulate */
    TQC_PREC_BF16 = 2,   /* dense steps on tcgen05, BF16 inputs, FP32 accumulate.  Does NOT meet the
                            1e-3 total-variation gate of the tensor-core forms on pseudo-physical
                            inputs (measured 1.2e-3 to 1.6e-3: operands keep 8 significant bits);
                            offered for speed comparisons, never chosen by TQC_PREC_AUTO */
    TQC_PREC_BF16X3 = 3, /* dense steps on tcgen05, split BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate */
    TQC_PREC_AUTO = 4    /* library's choice, per step: TF32 for a step that split BF16 would leave
                            bound by the tensor pipe (its MMA time above its HBM time), split BF16
                            for every other tensor-core step; CUDA-core steps stay FP32 */
};

/* contraction-order search (§III-E-1) */
enum {
    TQC_PLANNER_GREEDY = 0,      /* greedy pairwise merge on the predicted step time */
    TQC_PLANNER_EXHAUSTIVE = 1,  /* every contraction tree (m <= 9), best predicted time */
    TQC_PLANNER_LEARNED = 2,     /* candidates within 10x of the best analytic estimate, ranked
                                    by log(analytic seconds) + the learned MLP's output (a model
                                    trained on log(measured / analytic seconds)) */
    TQC_PLANNER_AUTO = 3         /* exhaustive for m <= 12, else greedy */
};

/* plan flags */
enum {
    TQC_FLAG_NO_RENORM = 1,      /* skip division by the total mass Z (Z still reported) */
    TQC_FLAG_REUSE = 2,          /* keep intermediates across tqc_contract calls (see there) */
    TQC_FLAG_NO_FUSE = 4,        /* run every step as its own kernel (no fused step pairs) */
    TQC_FLAG_NO_SMALLK = 8       /* CUDA-core steps with K = 1, 4 or 16 take the general
                                    64 x 64 .. 128 x 128 tiles instead of the small-K tile */
};

/*
 * One subcircuit tensor in the Pauli basis (§II-A: p_j^{e}, §III-B: a tensor
 * with one index per cut edge).
 *   n_out, out_qubits : bit k of the output index x is original qubit out_qubits[k]
 *   n_cut, cut_ids    : tensor axis d is cut edge cut_ids[d] (dim 4, order I,X,Y,Z);
 *                       cut ids of a network are 0..n_cuts-1, each used by exactly
 *                       two subcircuits
 *   cut_role          : per axis, 0 = this subcircuit measures the cut (upstream),
 *                       1 = it initialises the cut (downstream)
 *   dtype, data       : TQC_F64 or TQC_F32 host array, row-major
 *                       [c_0][c_1]...[c_{n_cut-1}][x], 4^n_cut * 2^n_out elements;
 *                       data == NULL for every subcircuit makes a shape-only
 *                       network (planning only, no device memory).
 */
typedef struct {
    int32_t n_out;
    const int32_t *out_qubits;
    int32_t n_cut;
    const int32_t *cut_ids;
    const int8_t *cut_role;
    int32_t dtype;
    const void *data;
} tqc_subcircuit;

/*
 * Validate the labels and build the network.  With data, copies every tensor
 * to the current CUDA device (synchronously); the caller keeps ownership of
 * its host arrays.  Fails with TQC_ERR_INVALID if output qubits do not
 * partition 0..n_qubits-1, if a cut id is out of range, appears other than
 * once upstream and once downstream, or joins a subcircuit to itself.
 */
TQC_API tqc_status tqc_network_create(int32_t n_qubits, int32_t n_sub, const tqc_subcircuit *subs,
                                      tqc_net_t *out);

/*
 * Replace the tensor data of subcircuit `sub` (same shape) from host memory,
 * stream-ordered on `cuda_stream` (asynchronous when host_data is pinned).
 * The network must have been created with data.
 */
TQC_API tqc_status tqc_network_upload(tqc_net_t net, int32_t sub, int32_t dtype, const void *host_data,
                                      void *cuda_stream);

/* Free the network's device copies.  Plans made from it must be destroyed first. */
TQC_API tqc_status tqc_destroy(tqc_net_t net);

typedef struct {
    int32_t use_free_mask;               /* 0 = every qubit free; 1 = the masks name the free
                                            qubits (none set = a single state) */
    uint64_t free_mask_lo, free_mask_hi; /* free qubits (bit q of lo = qubit q, of hi = q+64) */
    const uint8_t *fixed_bits;           /* n_qubits bytes, bit value of each non-free qubit;
                                            NULL = all zero; copied by tqc_plan */
    int32_t precision;                   /* TQC_PREC_* */
    int32_t planner;                     /* TQC_PLANNER_* */
    uint64_t mem_budget_bytes;           /* device bytes for operands, intermediates and the
                                            FP64 slice sum; 0 = unlimited.  A final step split
                                            along K (few tiles, long K loop) also keeps FP32
                                            partials of at most budget / 16 bytes (1 GiB when
                                            unlimited) */
    const char *costmodel_path;          /* learned cost model file (TQC_PLANNER_LEARNED) */
    int32_t autotune;                    /* 1 = time candidate tiles on first contract */
    int32_t n_order;                     /* optional forced contraction order: n_order pairs */
    const int32_t *order;                /* (a, b) per step; leaves are 0..m-1, step s makes m+s */
    int32_t n_sliced;                    /* optional forced sliced cuts (added to planner's) */
    const int32_t *sliced_cuts;
    int32_t flags;                       /* TQC_FLAG_* */
} tqc_plan_opts;

/* Fill defaults: every qubit free, TQC_PREC_AUTO, TQC_PLANNER_AUTO, no budget. */
TQC_API void tqc_plan_opts_default(tqc_plan_opts *opts);

/*
 * Plan the contraction (host only; no device work): contraction order
 * (§III-E-1), slicing of the most size-reducing cut edges until inputs, then
 * intermediates, fit the budget (§III-E-2), per-step kernel class, operand
 * precision and tensor layouts.  Two consecutive split-BF16 tensor-core
 * steps whose layouts line up (the first with K = 64 writing the row operand
 * of the second, K = 256 and N = 128; each 128 x 256 tile of the first
 * result is one 128-row tile of the second step's operand) are marked to run
 * as one kernel that keeps the intermediate on chip ("fuse" in
 * tqc_plan_describe: 1 on the first step, 2 on the second), unless
 * TQC_FLAG_NO_FUSE is set.
 */
TQC_API tqc_status tqc_plan(tqc_net_t net, const tqc_plan_opts *opts, tqc_plan_t *out);

/*
 * Plan totals.  flops = 2 * multiply-adds over all steps and slices (the
 * paper's cost unit, §III-C, counts the multiplications); bytes = algorithmic
 * HBM bytes (operands read once, results written once); any pointer may be NULL.
 */
TQC_API tqc_status tqc_plan_info(tqc_plan_t plan, double *flops, double *bytes, int32_t *n_slices,
                                 int32_t *n_steps);

/*
 * One step of a plan: log2 of the GEMM view C[M,N] = sum_K A[M,K] B[N,K]
 * (M = left free outputs x left open cuts, N = right ones, K = shared cuts),
 * the kernel class (0 = CUDA-core, 1 = tcgen05 tensor core) and operand type
 * (TQC_PREC_*).  Any pointer may be NULL.
 */
TQC_API tqc_status tqc_plan_step(tqc_plan_t plan, int32_t step, int32_t *log2_m, int32_t *log2_n,
                                 int32_t *log2_k, int32_t *kernel_class, int32_t *precision);

/*
 * Plan summary as JSON in buf (NUL-terminated, truncated to size).  Returns
 * the full length needed, excluding the NUL, or -1 on a bad handle.  Each
 * step lists its shape, class, precision, result layout, tile configuration
 * ("tile": CUDA-core 0 = 64 x 64, 1 = 128 x 128, 2 = 128 x 64, 3 = the
 * small-K tile; tcgen05 0 = 128 x 128, 1 = 128 x 64, 2 = 128 x 128 and
 * 3 = 128 x 256 with the direct epilogue), "ksplit" (K ranges run by
 * separate CTAs, 1 = none) and "kblk" (1 = its operands are stored
 * K-blocked, [K / 64][rows][64], for rows over 64 KB; fixed by the plan).
 * The first contract sets tiles and splits (0 and 1 before it); the
 * autotuner may change them.
 */
TQC_API int32_t tqc_plan_describe(tqc_plan_t plan, char *buf, int32_t size);

/*
 * Reconstruct the bin into caller-owned device memory d_out (2^F elements of
 * out_dtype, TQC_F32 or TQC_F64), stream-ordered on cuda_stream (a
 * cudaStream_t; NULL = legacy default stream).
 *   fixed_bits : NULL = the plan's bin; else n_qubits bytes giving new bit
 *                values of the non-free qubits (same free set).
 *   z_out      : NULL, or host pointer receiving the total mass Z (FP64); a
 *                non-NULL z_out synchronises the stream.
 * Steps: bin restriction and layout (ingest), the pairwise contractions,
 * FP64 sum over slices, renormalisation by Z.  The first call allocates the
 * plan's workspace.
 * Reuse across bins (plans made with TQC_FLAG_REUSE): the plan's workspace
 * keeps every leaf operand and intermediate of the previous call.  A call
 * whose bin differs only in the fixed bits of some subcircuits (same
 * tensors, same free set) re-ingests only those subcircuits' leaves and
 * recomputes only the steps that depend on them (not slice-dependent
 * tensors, which the slice loop rewrites); the last step always runs.
 * tqc_plan_describe reports what the last call kept.  Passing the plan to
 * tqc_contract_batch turns it off (its launches rewrite the workspace).
 * Without the flag every call recomputes every step.
 * Device-side failures: every wait of a tensor-core step is bounded; one that
 * gives up sets the plan's error word and its output is wrong.  The word is
 * read only by a call with a non-NULL z_out: that call returns
 * TQC_ERR_TIMEOUT if any call on the plan since the last such report gave up,
 * and clears the word.  Calls with z_out == NULL never report it.
 */
TQC_API tqc_status tqc_contract(tqc_plan_t plan, const uint8_t *fixed_bits, void *d_out, int32_t out_dtype,
                                double *z_out, void *cuda_stream);

/*
 * Arbitrary output states (§VII-C measures the reconstruction of a list of
 * one million arbitrary states): P(x) for each of n_states states, each an
 * n_qubits-bit integer (qubit q = bit q; n_qubits <= 64), scaled like
 * tqc_contract (2^{-|E|} / Z, or 2^{-|E|} with TQC_FLAG_NO_RENORM).
 *   plan     : made with an empty free set (use_free_mask = 1, both masks 0)
 *              and unsliced; its order and layouts serve every state
 *   states   : host array of n_states uint64_t, copied to the device each
 *              call (TQC_ERR_INVALID if a state has bits at or above n_qubits)
 *   d_out    : caller-owned device buffer, n_states elements of out_dtype
 *   z_out    : as in tqc_contract
 * Two forms, reported by tqc_plan_describe as "states_form": "fused" (one
 * kernel: a CTA contracts one state at a time in shared memory from per-node
 * tables T_j transposed to [x][cuts], built once per tensor version, FP32
 * arithmetic) when every single-state intermediate fits in shared memory;
 * "per-state" otherwise (the plan runs once per state through the ordinary
 * step kernels, with the state's bits as fixed bits; a host loop).  The
 * first call allocates the tables and a device copy of the list (grown when a
 * longer list comes); the list copy and the per-state loop make the call
 * synchronous with respect to the host.
 */
TQC_API tqc_status tqc_contract_states(tqc_plan_t plan, const uint64_t *states, int64_t n_states, void *d_out,
                                       int32_t out_dtype, double *z_out, void *cuda_stream);

/*
 * End-to-end form with host buffers: copies every subcircuit tensor from
 * host_tensors[j] (dtype in_dtype, NULL = unchanged) to the device and runs
 * tqc_contract.  When host_out is pinned host memory mapped into the device's
 * address space, the last kernel stores the 2^F results (out_dtype) straight
 * into it; otherwise they go to a plan-owned device buffer and are copied
 * into host_out.  Synchronises the stream.
 */
TQC_API tqc_status tqc_contract_host(tqc_plan_t plan, const void *const *host_tensors, int32_t in_dtype,
                                     void *host_out, int32_t out_dtype, double *z_out, void *cuda_stream);

/*
 * Many plans (independent networks of uneven sizes) in one persistent launch:
 * one kernel drains a device work list of every plan's ingest chunks and
 * step tiles (CUDA-core and tcgen05), each waiting, with a bounded wait, on
 * the counters of the items that produce its operands.  A plan's steps from
 * its first large one on (predicted to take at least the threshold of
 * tqc_batch_tail_threshold) run after that kernel as the ordinary step
 * kernels of tqc_contract, on four library-owned streams forked from
 * cuda_stream and joined back to it before the call returns (so the call
 * stays stream-ordered and capturable).  d_outs[i] receives
 * plan i's bin (FP32, renormalised with the plan's cached total mass).
 * Requirements: every plan was contracted once since its tensors last
 * changed, and none is sliced (TQC_ERR_UNSUPPORTED otherwise).  The first
 * call with a given (plans, outputs) list builds and uploads the work list
 * (allocates, synchronises); repeated calls with the same list only reset
 * the counters and launch, so they can be captured in a CUDA graph.  Calls
 * that overlap on the GPU share the work list and race.
 */
TQC_API tqc_status tqc_contract_batch(const tqc_plan_t *plans, void *const *d_outs, int32_t n,
                                      void *cuda_stream);

/* Synchronise `cuda_stream` and report the last batched launch:
 * TQC_ERR_TIMEOUT if one of its bounded device waits gave up (in the
 * persistent kernel, or in a large step launched after it). */
TQC_API tqc_status tqc_batch_status(void *cuda_stream);

/* Predicted step time (seconds, cost model of tqc_plan) from which a plan's
 * steps leave the persistent kernel of tqc_contract_batch and run as their
 * own launches after it: 0 = every step, a huge value = none; default 16e-6.
 * TQC_ERR_INVALID for a negative or NaN value. */
TQC_API tqc_status tqc_batch_tail_threshold(double seconds);

/* Kernel launches of one tqc_contract_batch call with the last list (the
 * persistent kernel plus the large steps' own launches) and the number of
 * steps that ran after it (tail_steps may be NULL).  TQC_ERR_INVALID before
 * any batch was launched. */
TQC_API tqc_status tqc_batch_launches(int64_t *launches, int64_t *tail_steps);

/* Fault-injection hook for tests: while enabled, batched launches carry one
 * extra item that waits on a counter nothing increments, so its bounded wait
 * must give up (about one second) and tqc_batch_status must report it. */
TQC_API tqc_status tqc_batch_inject_stall(int32_t enable);

/* Fault-injection hook for tests: while enabled, every tensor-core step
 * launched by tqc_contract or tqc_contract_noalloc has its first CTA skip
 * its first operand copy, so that CTA's MMA issuer gives up waiting (about
 * two seconds), drains, frees its tensor memory and sets the error word:
 * the call then reports TQC_ERR_TIMEOUT as described for each entry point.
 * Nothing faults; the output of such a call is wrong. */
TQC_API tqc_status tqc_step_inject_stall(int32_t enable);

/*
 * Per-step device timing (for roofline reporting).  enable = 1 makes every
 * following tqc_contract record a CUDA event pair, on the caller's stream,
 * around each pairwise-step launch; enable = 0 stops recording and clears
 * the records.  tqc_plan_step_time synchronises on the recorded events and
 * returns the mean duration (ms) and number of recorded launches of `step`.
 */
TQC_API tqc_status tqc_plan_profile(tqc_plan_t plan, int32_t enable);
TQC_API tqc_status tqc_plan_step_time(tqc_plan_t plan, int32_t step, double *mean_ms, int32_t *launches);

TQC_API tqc_status tqc_plan_destroy(tqc_plan_t plan);

/*
 * Allocation-free reconstruction.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory when they
 * reconstruct -- a process whose device memory is owned by another
 * framework's caching allocator or capped (MPS), a latency-critical loop in
 * which cudaMalloc/cudaFree would synchronise the device, or code whose
 * policy forbids touching the allocator.
 *
 * Same result as tqc_contract for the same plan and tensors, but every
 * intermediate lives in one file-scope device array of
 * tqc_noalloc_scratch_bytes() bytes (16 MiB), which every GPU that loads the
 * library holds until the process exits.  The call allocates nothing: it
 * takes the default tile of every step, never autotunes (whatever the plan's
 * autotune option) and never splits K.
 *   plan      : from tqc_plan; its network may be shape-only (data == NULL)
 *   d_tensors : m device pointers, caller-owned, subcircuit j in the layout of
 *               tqc_subcircuit.data, element type in_dtype (TQC_F64/TQC_F32)
 *   fixed_bits: as in tqc_contract (NULL = the plan's bin)
 *   d_out     : caller-owned device buffer of 2^F elements of out_dtype
 * Returns TQC_ERR_UNSUPPORTED, before any device work, when the plan needs
 * more scratch than the array holds.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race and corrupt each
 * other.  The call reads and changes none of the plan's or the network's
 * own device state, so tqc_contract on the same plan is unaffected.  The
 * first call on a device looks the array's address up with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Each call ends by copying its 4-byte error word into a host stack
 * variable, so it synchronises cuda_stream; it returns TQC_ERR_TIMEOUT when
 * a bounded wait of one of its tensor-core steps gave up (the output is then
 * wrong).
 */
TQC_API tqc_status tqc_contract_noalloc(tqc_plan_t plan, const void *const *d_tensors, int32_t in_dtype,
                                        const uint8_t *fixed_bits, void *d_out, int32_t out_dtype,
                                        void *cuda_stream);
TQC_API int64_t tqc_noalloc_scratch_bytes(void);

/*
 * Learned cost model (replaces the FLOP-count estimate of Eq.
 * classical_runtime, §V, which the paper finds consistently high).  A
 * multilayer perceptron, 3 hidden layers of 128 ReLU units, maps a plan's
 * TQC_PLAN_FEATURES features (tqc_plan_features) to a log-time target.  The
 * learned planner (TQC_PLANNER_LEARNED) reads its output as the log of the
 * plan's measured over its analytic contraction time, i.e. a correction to
 * the planner's own estimate.  Forward, backward and Adam run in the
 * library's CUDA kernels on the current device (FP32); calls synchronise.
 *
 * Parameter layout (flat): W1 [F x 128], b1 [128], W2 [128 x 128], b2,
 * W3 [128 x 128], b3, W4 [128 x 1], b4; rows of X are samples, Y = X W + b.
 */
#define TQC_PLAN_FEATURES 32
typedef struct tqc_costmodel *tqc_costmodel_t;

/* New model with He-uniform weights from a seeded generator, zero biases. */
TQC_API tqc_status tqc_costmodel_create(int32_t n_features, uint64_t seed, tqc_costmodel_t *out);
TQC_API tqc_status tqc_costmodel_destroy(tqc_costmodel_t model);
/* Copy the parameters out (h_out == NULL: only report the count in *n). */
TQC_API tqc_status tqc_costmodel_params(tqc_costmodel_t model, float *h_out, int32_t *n);
TQC_API tqc_status tqc_costmodel_set_params(tqc_costmodel_t model, const float *h_in, int32_t n);
/* Mean squared error of the raw network on (X [n x F], t [n]) and its
 * gradient w.r.t. the flat parameters (no standardisation applied). */
TQC_API tqc_status tqc_costmodel_grad(tqc_costmodel_t model, const float *h_X, const float *h_t, int32_t n,
                                      float *h_grad, float *h_loss);
/* Fit log-times: standardises features and labels (statistics kept with the
 * model), then `epochs` passes of Adam (lr, beta 0.9/0.999) over shuffled
 * minibatches; *final_loss = mean standardised MSE of the last epoch. */
TQC_API tqc_status tqc_costmodel_train(tqc_costmodel_t model, const float *h_X, const float *h_logt, int32_t n,
                                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *final_loss);
/* Predicted log-times (seconds) of n feature rows. */
TQC_API tqc_status tqc_costmodel_predict(tqc_costmodel_t model, const float *h_X, int32_t n, float *h_logt);
TQC_API tqc_status tqc_costmodel_save(tqc_costmodel_t model, const char *path);
TQC_API tqc_status tqc_costmodel_load(const char *path, tqc_costmodel_t *out);

/* The TQC_PLAN_FEATURES features of a plan (n must be >= TQC_PLAN_FEATURES). */
TQC_API tqc_status tqc_plan_features(tqc_plan_t plan, float *out, int32_t n);
/*
 * Candidate contraction orders the learned planner ranks: the optima of the
 * time, multiply-add and byte models, the greedy order, then seeded random
 * trees.  orders receives up to max_n orders of n_sub-1 (a, b) pairs each in
 * the SSA form of tqc_plan_opts.order; *n_out = number written.
 */
TQC_API tqc_status tqc_plan_candidates(tqc_net_t net, const tqc_plan_opts *opts, int32_t max_n, int32_t *orders,
                                       int32_t *n_out);

/* Thread-local description of the last error ("" if none). */
/*
 * Heavy state selection (§IV, Alg. heavy_state_selection): reconstruct only
 * the product of a few heavy output states per subcircuit.
 */
/* The L2 norm over all cut assignments of every output state of subcircuit
 * `sub`: d_norms[i] = sqrt(sum_e T_sub[e][i]^2), i in [0, 2^{n_out}).
 * d_norms: device, FP64, 2^{n_out} entries, caller-owned; stream-ordered.
 * Deterministic: the partial sums are added in a fixed order.  When the
 * output states alone cannot fill the GPU the sum is split over the cut
 * assignments, with a stream-ordered scratch allocation (cudaMallocAsync) of
 * a few MB for the partials. */
TQC_API tqc_status tqc_hss_norms(tqc_net_t net, int32_t sub, double *d_norms, void *cuda_stream);
/* Select heavy states: norms on the device, then every subcircuit is seeded
 * with its heaviest state and states are added in descending norm (ties:
 * lower subcircuit, then lower index) while the product of the per-subcircuit
 * counts is below s_max.  Out (host): counts[m]; states (capacity
 * states_cap) = each subcircuit's selected state indices, ascending,
 * concatenated in subcircuit order; *n_states = the product of the counts.
 * Synchronous.  TQC_ERR_INVALID if states_cap is too small. */
TQC_API tqc_status tqc_hss_select(tqc_net_t net, int64_t s_max, int32_t *counts, int32_t *states,
                                  int64_t states_cap, int64_t *n_states);
/* A new network whose subcircuit j keeps only the output states
 * states[o_j .. o_j + counts[j]) (ascending indices into its 2^{n_out} states;
 * o_j = counts[0] + ... + counts[j-1]), padded with zero rows to 2^{k_j},
 * k_j = ceil(log2 counts[j]).  Its outputs are the selection indices:
 * subcircuit j's k_j bits follow those of subcircuits 0..j-1 (at least one
 * bit in total).  Cuts and roles are unchanged; the rows are gathered on the
 * device (synchronous).  Contract it with TQC_FLAG_NO_RENORM and divide by
 * the source network's total mass to get the product states' probabilities;
 * padded entries are zero.  Destroy with tqc_destroy. */
TQC_API tqc_status tqc_network_select(tqc_net_t net, const int32_t *counts, const int32_t *states, tqc_net_t *out);

/*
 * Cut finder (§VI): Greedy Graph Growing (Alg. 2) over the circuit's
 * two-qubit gates, merging the partitions joined by the edge of least
 * merging cost (Alg. 3, Table I) until none is valid; one-qubit gates then
 * join an adjacent two-qubit gate.  Among the partitions found for
 * thresholds K_t = 1..k_sweep_max (or the one given) it returns the one of
 * least T = T_QPU + T_classical (Eq. cut_objective): T_QPU by Eq.
 * qpu_runtime, T_classical the planner's estimated time to contract the
 * resulting network for the bin of the lowest cost_free_qubits qubits (the
 * analytic step-time model, times exp of the learned cost model's output
 * when costmodel_path is given, in place of Eq. classical_runtime's FLOP
 * count over FLOP/s).  Host only (the learned model runs on the device).
 *   gate_qubits : n_gates x 2 qubit ids in time order; second = -1 for a
 *                 one-qubit gate
 *   gate_part   : out, n_gates subcircuit ids (numbered by first gate); a
 *                 wire is cut wherever consecutive gates on it sit in
 *                 different subcircuits (upstream end: the earlier gate's);
 *                 a wire without two-qubit gates joins subcircuit 0, whose
 *                 width may then exceed w_max (result->max_width says)
 * Readings of what the paper leaves open: a subcircuit's width is its number
 * of wire segments (a wire that leaves and re-enters comes back on a new
 * qubit) and its size its number of two-qubit gates; the contraction edges
 * of two neighbouring partitions are the distinct cuts touching either;
 * every merging cost is recomputed after each merge and ties go to the
 * lowest (earlier gate, later gate) edge; shots = 2^width limited to
 * [2^shots_log2_min, 2^shots_log2_max]; depth = layers of the subcircuit's
 * gates scheduled as early as possible.
 */
typedef struct {
    int32_t w_max;            /* most qubits of a subcircuit (hard limit) */
    int32_t s_max;            /* most two-qubit gates of a subcircuit (hard limit) */
    int32_t k_t;              /* contraction-edge threshold (soft); <= 0: sweep 1..k_sweep_max */
    int32_t k_sweep_max;
    double q_max;             /* merging-cost cutoff; <= 0: none */
    double t_gate, t_meas;    /* seconds per gate layer and per measurement (Eq. qpu_runtime) */
    int32_t shots_log2_min, shots_log2_max;
    int32_t n_qpus;           /* QPUs running subcircuits in parallel (T_QPU is divided by it) */
    int32_t cost_free_qubits; /* T_classical: the bin of this many lowest qubits (<= 40) */
    int32_t precision;        /* of the plan estimating T_classical */
    const char *costmodel_path; /* learned cost model for T_classical, or NULL */
} tqc_cut_opts;

typedef struct {
    int32_t n_sub, n_cuts, k_t, max_width;
    double t_qpu, t_classical, t_total;  /* seconds */
    double cutqc_mults, tensorqc_mults;  /* per state: brute force 4^|E| (m-1); the plan's order on one state */
} tqc_cut_result;

/* Defaults: w_max 16, no gate limit, K_t swept 1..16, no Q_max, t_gate 1e-7 s,
 * t_meas 1e-6 s, shots 2^10..2^20, 10 QPUs (§VII-A), a 2^20-state bin, AUTO. */
TQC_API void tqc_cut_opts_default(tqc_cut_opts *opts);
TQC_API tqc_status tqc_find_cuts(int32_t n_qubits, int32_t n_gates, const int32_t *gate_qubits,
                                 const tqc_cut_opts *opts, int32_t *gate_part, tqc_cut_result *result);

/*
 * Classical cost of a plan against the brute-force reconstruction (§III-C;
 * §VIII, Fig. cost_ratio compares CutQC's brute force with TensorQC's
 * contraction in scalar multiplications).
 */
typedef struct {
    double cutqc_mults_per_state;    /* 4^|E| (m - 1): every cut assignment, m - 1 products each */
    double tensorqc_mults_per_state; /* the plan's contraction order on a single state */
    double ratio;                    /* cutqc / tensorqc, per state */
    double plan_mults;               /* the plan itself: every slice and every state of its bin */
    double plan_mults_per_state;     /* plan_mults / 2^F (shared work across the bin) */
    int32_t k_max;                   /* most contraction edges (inner + outer cuts) of a single-state step */
    double tn_upper_bound;           /* 4^{k_max} m (Eq. tn_upper_bound) */
} tqc_cost_report;
TQC_API tqc_status tqc_plan_cost_report(tqc_plan_t plan, tqc_cost_report *out);

TQC_API const char *tqc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TQC_H_ */

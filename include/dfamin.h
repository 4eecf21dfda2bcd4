/*
 * dfamin: GB300 (sm_103a) DFA minimizer - public C ABI.
 *
 * Computes the coarsest partition of the states of a complete DFA that refines {F, Q\F} and is
 * stable under the transition function, i.e. language equivalence of states (arXiv 2410.22764,
 * Sec. 2 problem statement and Definition of a DFA).  The initial state is not an input and
 * unreachable states are not removed: every state is classified (Sec. 2: the refinement
 * algorithms take every state to be reachable; removing unreachable states is a separate
 * pre-processing step, see dfamin_reachable).  The method is signature-based partition refinement
 * (Alg. sortPR, Sec. 3.3), optionally on the partial transitive closure A' of Alg. transPR
 * (Sec. 3.4), which has the same state equivalence as A.
 *
 * Data conventions (all calls):
 *   n       number of states, 1 <= n <= 2^30.  States are 0..n-1.
 *   k       number of letters, k >= 0.  Letters are 0..k-1.  n*k < 2^40.
 *   delta   int32 [n*k], STATE-MAJOR: delta[s*k + a] = delta(s, a), each in [0, n).  (The paper
 *           stores delta[a][q] letter-major, Sec. 2 "Representation"; the library may use any
 *           layout internally.)  May be NULL when k == 0.
 *   accept  uint32 bitmap [(n+31)/32]: state s is accepting iff (accept[s>>5] >> (s&31)) & 1.
 *   out_block int32 [n]: canonical block ids.  The id of a block is the number of blocks whose
 *           smallest state is smaller than its own smallest state (first-occurrence order over
 *           s = 0..n-1), so block ids are 0..nblocks-1 and out_block[0] == 0.
 *
 * Memory and streams: every array pointer is a DEVICE pointer (cudaMalloc / torch CUDA memory)
 * owned by the caller.  Calls are asynchronous on `stream` (NULL = legacy default stream): they
 * validate host-side arguments, enqueue work and return.  Outputs are valid once the stream has
 * reached that point.  The inputs are never modified.  Nothing here synchronises the stream.
 *
 * Errors: host-detectable errors (bad sizes, NULL pointers, workspace too small, launch
 * failure) are returned synchronously and nothing is enqueued.  Errors found on the device
 * (a delta entry out of range, a bounded wait that ran out, no convergence within max_passes)
 * are written to the `status` output (DFAMIN_OK when fine); in that case out_block is not
 * meaningful and *nblocks is set to minus the status code.
 */
#ifndef DFAMIN_H
#define DFAMIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same handle as cudaStream_t; declared opaquely so this header needs no CUDA headers. */
typedef struct CUstream_st *dfamin_stream_t;

typedef enum {
    DFAMIN_OK = 0,
    DFAMIN_EINVAL = 1,      /* bad argument, or (on device) a delta entry outside [0, n) */
    DFAMIN_ENOMEM = 2,      /* workspace too small / internal allocation failed */
    DFAMIN_ECUDA = 3,       /* a CUDA runtime call failed */
    DFAMIN_ETIMEOUT = 4,    /* a bounded device-side wait (CTA barrier) ran out */
    DFAMIN_ENOCONVERGE = 5, /* max_passes reached before the partition was stable */
    DFAMIN_EPROBE = 6       /* hash-table probe sequence exhausted (table full) */
} dfamin_status;

/* closure */
#define DFAMIN_CLOSURE_OFF 0   /* plain refinement on A (Alg. sortPR semantics) */
#define DFAMIN_CLOSURE_ON 1    /* refinement on the closed DFA A' of Alg. transPR */

/* algorithm */
#define DFAMIN_ALG_SIGNATURE 0 /* signature refinement, Alg. sortPR (Sec. 3.3): a block may split
                                  into many blocks per round (default) */
#define DFAMIN_ALG_LEADER 1    /* leader election, Alg. 2 naivePR (Sec. 3.2): per round, the states
                                  of a block that differ from its leader move, together, to one new
                                  block led by the smallest of them; rounds run until one changes
                                  nothing (the final, unchanged round is counted).  With the closure
                                  this is transPR exactly as Alg. transPR runs it (naivePR on A') */

/* flags */
#define DFAMIN_FLAG_KEEP_IDENTITY 1u  /* closure: build every column of A'.  By default letters
                                         whose delta is the identity get no closure columns, and
                                         a letter stops getting levels once level i equals level
                                         i-1 (every later level would repeat it); repeated
                                         columns change no partition and no pass count */
#define DFAMIN_FLAG_HASH_BLOCK_ONLY 2u /* testing: hash only the old block id (forces collisions
                                         that the full-tuple check must resolve) */
#define DFAMIN_FLAG_HASH_CONSTANT 4u   /* testing: constant hash (every group collides) */
#define DFAMIN_FLAG_TRACE 8u           /* record per-phase device timestamps (see below) */
#define DFAMIN_FLAG_FULL_ROUNDS 16u    /* testing and measurement: every signature round re-reads
                                         every state's successors.  By default a round that
                                         follows a signature round in which few states moved is
                                         incremental: it skips the blocks that cannot split (a
                                         block whose members' successors all lie in blocks that
                                         did not split in the previous round keeps its members;
                                         same partition, same pass count) */
#define DFAMIN_FLAG_BATCH_FOUR_CTAS 64u /* batches (tuning): run the batch kernel built for four
                                         resident CTAs per SM (64 registers a thread) instead of
                                         three (80 registers); results are the same */
#define DFAMIN_FLAG_INCREMENTAL_ROUNDS 32u /* testing: every signature round that follows another
                                         one is incremental, however many states moved (the
                                         default chooses by that number).  FULL_ROUNDS wins if
                                         both are set */
#define DFAMIN_FLAG_MASKED_ROUNDS 128u /* testing: every signature round that follows another
                                         one is letter-masked (compile-time alphabets k <= 8, no
                                         closure): each leader marks the letters whose entry names
                                         a block that split in the previous round, and members
                                         gather only those letters (the others cannot differ from
                                         the leader's).  By default a round is masked when members
                                         outnumber leaders or few states moved, and the partition
                                         has more than a few thousand blocks.  Same partition, same
                                         pass count.  FULL_ROUNDS and INCREMENTAL_ROUNDS win if
                                         set */

/* Phase trace.  With DFAMIN_FLAG_TRACE the workspace grows by DFAMIN_TRACE_BYTES, and the last
 * DFAMIN_TRACE_BYTES of the required workspace receive int64 values: [0] = number of records,
 * then records (tag, t_ns) with tag = (pass << 8) | phase and t_ns the device global timer
 * when the phase ended.  Phases: 0 start, 1 validation, 2 initial partition, 3 one closure
 * level, 4 leaders' signatures, 5 members' regrouping, 6 moves applied, 7 leader count,
 * 8 canonical ids written.  Records beyond capacity are counted but not stored. */
#define DFAMIN_TRACE_BYTES 262144

typedef struct {
    int32_t closure;     /* DFAMIN_CLOSURE_OFF or DFAMIN_CLOSURE_ON */
    int32_t max_passes;  /* cap on signature passes; 0 = n + 1 */
    uint32_t flags;      /* DFAMIN_FLAG_* */
    int32_t ctas;        /* 0 = automatic; otherwise number of CTAs for one DFA (tuning) */
    int32_t smem_states; /* 0 = automatic; largest n solved by one CTA (up to 8192 states
                            entirely in shared memory, up to 65535 with 16-bit block ids in
                            shared memory and the group table in global memory) */
    int32_t team_states; /* batches: 0 = automatic; states per CTA when sizing a DFA's team */
    int32_t algorithm;   /* DFAMIN_ALG_SIGNATURE (default) or DFAMIN_ALG_LEADER */
    int32_t barrier_timeout_us; /* 0 = default bound on every wait of a CTA for the other CTAs
                            of its team (4 s for one DFA, 30 s in batches); otherwise that bound
                            in microseconds.  A wait that runs out ends the call with status
                            DFAMIN_ETIMEOUT (every CTA leaves at its next barrier; the context
                            stays usable).  Meant for tests of that failure path: a bound of a
                            few microseconds makes a multi-CTA call fail without any fault.
                            One-CTA calls (small DFAs) have no such wait */
    int32_t closure_columns; /* closure: 0 = build every column (floor(log2 n) levels of every
                            letter); otherwise at most this many columns, level by level, and the
                            workspace shrinks to match.  Any subset of the closed alphabet gives
                            the same state equivalence (every added letter is a word over the
                            original alphabet), so fewer columns never change the partition, only
                            the number of passes (between the full closure's and the plain
                            count) */
} dfamin_options;

/* Fills *opt with the defaults (closure off, automatic tuning). */
void dfamin_default_options(dfamin_options *opt);

/*
 * dfamin_minimize - minimize one DFA (Sec. 2 problem; Alg. sortPR refinement, Sec. 3.3).
 * nblocks: device int32 scalar, receives the number of blocks (or -status on a device error).
 * Uses a workspace owned by the library (one per device and stream, grown on demand with
 * cudaMalloc, which may synchronise the device when it grows).  Closure off.
 */
dfamin_status dfamin_minimize(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                              int32_t *out_block, int32_t *nblocks, dfamin_stream_t stream);

/*
 * dfamin_workspace_size - bytes of device workspace dfamin_minimize_ex needs for (n, k, opt).
 */
dfamin_status dfamin_workspace_size(int32_t n, int32_t k, const dfamin_options *opt,
                                    size_t *bytes);

/*
 * dfamin_minimize_ex - as dfamin_minimize, with options and a caller-owned workspace.
 *   opt        NULL = defaults.  closure = ON runs the refinement on A' (Alg. transPR,
 *              Sec. 3.4): columns delta^T(., a^(2^i)) for i = 1..floor(log2 n) are built by
 *              pointer doubling and appended to every state's signature.
 *   workspace  device memory of at least dfamin_workspace_size() bytes, 256-byte aligned,
 *              any contents; the call owns it until the stream passes the call.  Calls that
 *              overlap on the GPU must not share a workspace.
 *   passes     device int32 scalar or NULL: number of signature passes executed.  A pass is
 *              one refinement round; the loop stops after a pass that left the block count
 *              unchanged, or once every block is a singleton (0 passes if {F, Q\F} is already
 *              discrete).
 *   status     device int32 scalar or NULL: DFAMIN_OK or the device-detected error.
 */
dfamin_status dfamin_minimize_ex(int32_t n, int32_t k, const int32_t *delta,
                                 const uint32_t *accept, int32_t *out_block, int32_t *nblocks,
                                 const dfamin_options *opt, void *workspace,
                                 size_t workspace_bytes, int32_t *passes, int32_t *status,
                                 dfamin_stream_t stream);

/*
 * dfamin_minimize_from_host - the same minimization as dfamin_minimize_ex, end to end from HOST
 * arrays: the rows and the bitmap are read from host memory and the labels and scalars are
 * written back to it, all in stream order on `stream`.
 *   h_delta     host int32 [n*k] (state-major, as for dfamin_minimize_ex); h_accept host uint32
 *               bitmap [(n+31)/32]; h_out_block host int32 [n] (canonical labels);
 *   h_scalars   host int32 [3]: nblocks (or -status), passes, status.
 *   workspace   DEVICE memory of dfamin_minimize_from_host_workspace_size() bytes, 256-byte
 *               aligned: the device copies of the inputs and outputs and the workspace of the
 *               minimization.
 * With page-locked host arrays (cudaHostAlloc, cudaHostRegister) the call is asynchronous and
 * moves data with no separate copy where it can: the bitmap is copied first, then the first
 * round reads every row straight from host memory (its only input besides the bitmap) while it
 * computes, storing the device copy that later rounds read, and the last pass writes the labels
 * and the scalars straight to host memory.  (That applies to DFAs solved by the multi-CTA
 * kernel with 1..8 letters and no closure; in every other case, and for pageable host arrays,
 * the arrays are copied before and after the kernel on the stream, and pageable arrays make the
 * call return only when its copies are done.)  The host arrays must stay valid, and h_delta
 * unchanged, until the stream has passed the call.
 */
dfamin_status dfamin_minimize_from_host_workspace_size(int32_t n, int32_t k,
                                                      const dfamin_options *opt, size_t *bytes);
dfamin_status dfamin_minimize_from_host(int32_t n, int32_t k, const int32_t *h_delta,
                                        const uint32_t *h_accept, int32_t *h_out_block,
                                        int32_t *h_scalars, const dfamin_options *opt,
                                        void *workspace, size_t workspace_bytes,
                                        dfamin_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Batches: many DFAs minimized in one persistent launch (each exactly as dfamin_minimize_ex
 * would: Alg. sortPR rounds, Sec. 3.3, optionally on the closed DFA of Alg. transPR, Sec. 3.4).
 *
 * A plan holds the host-side schedule for one shape of batch (the per-DFA sizes) and a small
 * device table (allocated at creation); launches with the same plan can be repeated and
 * captured in a CUDA graph.  Data of a batch of `count` DFAs, DFA i having n_i states and k_i
 * letters:
 *   state_off  HOST int64 [count+1], state_off[0] = 0, state_off[i+1] - state_off[i] = n_i >= 1
 *   k          HOST int32 [count], k_i >= 0
 *   delta      device int32, the DFAs' state-major tables concatenated in order (DFA i starts at
 *              sum_{j<i} n_j k_j); successor ids are LOCAL to their DFA (in [0, n_i))
 *   accept     device uint32 bitmap over the concatenated states: state s of DFA i is bit
 *              state_off[i] + s (LSB first)
 *   out_block  device int32 [state_off[count]]: canonical ids, local to each DFA
 *   nblocks, passes, status  device int32 [count] (passes and status may be NULL); a DFA with a
 *              device-detected error gets status != 0 and nblocks = -status, others are unaffected
 * The options of the plan apply to every DFA (closure, max_passes, flags).  For batches,
 * opt->smem_states is the largest n solved by one CTA in shared memory, opt->team_states the
 * states per CTA when sizing a larger DFA's team, opt->ctas a cap on the grid.
 * ------------------------------------------------------------------------------------------ */
typedef struct dfamin_batch_plan_s *dfamin_batch_plan;

dfamin_status dfamin_batch_plan_create(int32_t count, const int64_t *state_off, const int32_t *k,
                                       const dfamin_options *opt, dfamin_batch_plan *plan);
/* Plan creation and destruction use stream-ordered allocation on a library stream and never
 * wait for work on other streams.  Destroying a plan releases its device table after the most
 * recent launch that used it has completed (in stream order); a caller that launches one plan
 * on several streams at once must let those launches complete before destroying it.  A launch
 * captured into a CUDA graph is not tracked: the plan must outlive every replay of the graph. */
dfamin_status dfamin_batch_plan_destroy(dfamin_batch_plan plan);

/* Bytes of device workspace a launch with this plan needs (caller-owned, 256-byte aligned). */
dfamin_status dfamin_batch_workspace_size(dfamin_batch_plan plan, size_t *bytes);

/* Schedule facts: CTAs of the launch, team tickets, total states and transitions. */
dfamin_status dfamin_batch_plan_info(dfamin_batch_plan plan, int32_t *grid, int64_t *tickets,
                                     int64_t *states, int64_t *transitions);

/* Enqueue the minimization of every DFA of the plan's batch on `stream`; asynchronous.
 *   delta     concatenated int32 rows, successor ids LOCAL to each DFA (DFA i's rows start at
 *             sum_{j<i} n_j*k_j); accept one bitmap, bit state_off[i] + s for state s of DFA i.
 *   out_block concatenated [state_off[count]], canonical ids local to each DFA.
 *   nblocks, passes, status  device int32 [count] (passes and status may be NULL); a DFA with a
 *             device error gets status != 0 and nblocks = -status, the others are unaffected. */
dfamin_status dfamin_batch_plan_run(dfamin_batch_plan plan, const int32_t *delta,
                                    const uint32_t *accept, int32_t *out_block, int32_t *nblocks,
                                    int32_t *passes, int32_t *status, void *workspace,
                                    size_t workspace_bytes, dfamin_stream_t stream);

/*
 * dfamin_minimize_batch - one-shot form of the batch (no plan object): the schedule is computed
 * on the host for this call and its descriptor table is copied into the head of the caller's
 * workspace (a copy from pageable memory: the call returns once it is staged), so the call
 * allocates nothing.  state_off [num_dfas+1], k [num_dfas] and delta_off [num_dfas+1] (the
 * prefix of n_i*k_i, may be NULL as it is implied) are HOST arrays, because the schedule needs
 * the sizes; every other array is a device array with the layout of dfamin_batch_plan_run.
 * Launches that repeat one batch shape should use a plan (scheduled once, graph-capturable).
 * This one-shot call cannot be captured into a CUDA graph (its table copy reads host memory that
 * is gone once the call returns): on a capturing stream it returns DFAMIN_EINVAL and enqueues
 * nothing.
 */
dfamin_status dfamin_minimize_batch_workspace_size(int32_t num_dfas, const int64_t *state_off,
                                                   const int32_t *k, const dfamin_options *opt,
                                                   size_t *bytes);
dfamin_status dfamin_minimize_batch(int32_t num_dfas, const int64_t *state_off, const int32_t *k,
                                    const int64_t *delta_off, const int32_t *delta,
                                    const uint32_t *accept, int32_t *out_block, int32_t *nblocks,
                                    const dfamin_options *opt, void *workspace,
                                    size_t workspace_bytes, int32_t *status,
                                    dfamin_stream_t stream);

/*
 * dfamin_minimize_static - the same minimization as dfamin_minimize_ex, for callers that cannot
 * allocate device memory: for example a plugin or an embedded runtime whose host owns the whole
 * device-memory budget, or a latency-critical path where cudaMalloc's implicit device-wide
 * synchronisation is not acceptable.  It takes no workspace: it runs in a scratch array of
 * DFAMIN_STATIC_SCRATCH_BYTES that the library places in device memory as a file-scope static
 * variable, so every GPU that loads the library holds that array until the process exits.  The
 * paper has no counterpart; it is an engineering addition to the boundary.
 *   Limit     problems whose dfamin_workspace_size(n, k, opt) exceeds
 *             DFAMIN_STATIC_SCRATCH_BYTES are rejected with DFAMIN_ENOMEM before anything is
 *             enqueued (for k = 4 that is n of about one million states).
 *   Set-up    the first call on a device looks up the array's device address (with that device
 *             current) and caches it; make that first call before any stream capture.
 *   Sharing   all calls on a device share the one array and it keeps the last call's contents
 *             (the call clears what must start at zero).  Calls whose work overlaps on the GPU
 *             (other streams, other host threads) race on it: serialise them.
 *   Allocation  none: no cudaMalloc, cudaFree or other allocating routine is called.
 * The other arguments are those of dfamin_minimize_ex.
 */
#define DFAMIN_STATIC_SCRATCH_BYTES (64u << 20)
dfamin_status dfamin_minimize_static(int32_t n, int32_t k, const int32_t *delta,
                                     const uint32_t *accept, int32_t *out_block,
                                     int32_t *nblocks, const dfamin_options *opt,
                                     int32_t *passes, int32_t *status, dfamin_stream_t stream);


/*
 * Reachability and the minimal DFA (Sec. 2: minimizing a DFA merges indistinguishable states and
 * deletes the states unreachable from the initial state q0; the paper's refinement algorithms
 * assume the deletion was done as a pre-processing step).  The paper prints no algorithm for
 * these steps; they are plain definitions.
 *
 * dfamin_reachable - states reachable from q0 by some word.
 *   out_newid  int32 [n]: the rank of s among the reachable states in increasing state order
 *              (an order-preserving renumbering), or -1 if s is unreachable.
 *   out_delta  int32 [n*k] or NULL: the sub-DFA induced by the reachable states, renumbered:
 *              out_delta[newid[s]*k + a] = newid[delta(s, a)]; the first count*k entries are
 *              written.
 *   out_accept uint32 bitmap [(n+31)/32] or NULL: bit newid[s] is set iff s accepts (the
 *              whole bitmap is cleared first).
 *   count      device int32 or NULL: number of reachable states (or -status on a device error).
 *   status     device int32 or NULL: DFAMIN_OK, or DFAMIN_EINVAL if a row of a reachable state
 *              holds an entry outside [0, n) (rows of unreachable states are not read), or
 *              DFAMIN_ETIMEOUT.
 *   workspace  device, 256-byte aligned, dfamin_reach_workspace_size(n) bytes.
 * Breadth-first search in which a thread keeps following the states it claims (far along a
 * chain, briefly once the frontier grows); a chain of L states takes about L/256
 * barrier-separated levels and L dependent loads, so long chains are latency-bound.
 */
dfamin_status dfamin_reach_workspace_size(int32_t n, size_t *bytes);
dfamin_status dfamin_reachable(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                               int32_t q0, int32_t *out_newid, int32_t *out_delta,
                               uint32_t *out_accept, int32_t *count, int32_t *status,
                               void *workspace, size_t workspace_bytes, dfamin_stream_t stream);

/*
 * dfamin_quotient - the quotient automaton of a partition (Sec. 2, combining states).
 *   block      int32 [n]: class of every state, any ids in [0, n) (for example out_block of
 *              dfamin_minimize_ex).  The partition must be stable under delta for the result to
 *              be the quotient; the class of delta(rep, a) is taken from the class's smallest
 *              member rep.
 *   newid      int32 [n] or NULL: out_newid of dfamin_reachable on the same DFA; only states
 *              with newid[s] >= 0 are kept (q0 must be one of them).  NULL keeps every state.
 *   out_delta  int32 [n*k] capacity: out_delta[B*k + a] for the nstates output classes, which
 *              are numbered in the order of their smallest kept member.
 *   out_accept uint32 bitmap [(n+31)/32] (cleared first): bit B set iff class B accepts.
 *   nstates    device int32: number of classes (or -status); out_q0 device int32 or NULL: the
 *              class of q0; status device int32 or NULL.
 *   workspace  device, 256-byte aligned, dfamin_quotient_workspace_size(n) bytes.
 */
dfamin_status dfamin_quotient_workspace_size(int32_t n, size_t *bytes);
dfamin_status dfamin_quotient(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                              const int32_t *block, int32_t q0, const int32_t *newid,
                              int32_t *out_delta, uint32_t *out_accept, int32_t *nstates,
                              int32_t *out_q0, int32_t *status, void *workspace,
                              size_t workspace_bytes, dfamin_stream_t stream);

/*
 * dfamin_minimal_dfa - the minimal DFA of (delta, accept, q0): dfamin_reachable, the
 * refinement of dfamin_minimize_ex (with `opt`) on the whole DFA, and dfamin_quotient restricted
 * to the reachable states, enqueued on `stream` with no host synchronisation.  Classes of the
 * whole DFA restricted to the reachable states are the classes of the reachable sub-DFA
 * (equivalence of two states depends only on the states reachable from them).
 *   out_delta   int32 [n*k] capacity, out_accept uint32 [(n+31)/32]: the minimal DFA, states
 *               numbered in the order of their smallest reachable member.
 *   out_scalars device int32 [5]: nstates (or -status), q0 of the minimal DFA, number of
 *               reachable states, refinement passes, status (first error of any stage).
 *   workspace   device, 256-byte aligned, dfamin_minimal_dfa_workspace_size(n, k, opt) bytes.
 */
dfamin_status dfamin_minimal_dfa_workspace_size(int32_t n, int32_t k, const dfamin_options *opt,
                                                size_t *bytes);
dfamin_status dfamin_minimal_dfa(int32_t n, int32_t k, const int32_t *delta,
                                 const uint32_t *accept, int32_t q0, const dfamin_options *opt,
                                 int32_t *out_delta, uint32_t *out_accept, int32_t *out_scalars,
                                 void *workspace, size_t workspace_bytes, dfamin_stream_t stream);

/*
 * dfamin_lts_determinize - LTS -> DFA front end (Sec. 4.1, VLTS paragraph): the powerset construction
 * from s0 makes the LTS deterministic; every subset state accepts; one extra non-accepting state
 * (bottom) receives every missing transition and loops on every label.  HOST code on HOST
 * arrays (it prepares input for the device calls; it runs on the calling thread and uses no
 * GPU).
 *   n, nlabels, m   states, labels and transitions of the LTS; transition i is
 *                   src[i] -lbl[i]-> dst[i] (duplicates allowed).
 *   max_states      capacity of the outputs in DFA states (bottom included).
 *   out_delta       host int32 [max_states*nlabels], state-major; out_accept host uint32 bitmap
 *                   [(max_states+31)/32]; *out_n = number of DFA states.
 * Numbering: subsets in the order a FIFO breadth-first search discovers them, labels taken in
 * increasing order; {s0} is state 0; bottom is state *out_n - 1.
 * Returns DFAMIN_EINVAL for an entry out of range, DFAMIN_ENOMEM (and *out_n = -1) when more
 * than max_states states are needed.
 */
dfamin_status dfamin_lts_determinize(int32_t n, int32_t nlabels, int64_t m, const int32_t *src,
                                     const int32_t *lbl, const int32_t *dst, int32_t s0,
                                     int32_t max_states, int32_t *out_delta,
                                     uint32_t *out_accept, int32_t *out_n);

/* Text of the last CUDA runtime failure seen by the library on the calling thread ("" if
 * none); meant for diagnostics after DFAMIN_ECUDA / DFAMIN_ENOMEM.  Thread-local storage. */
const char *dfamin_last_cuda_error(void);

/* Human-readable name of a status code (static string). */
const char *dfamin_status_string(dfamin_status s);

#ifdef __cplusplus
}
#endif

#endif /* DFAMIN_H */

// Device code of the refinement (shared by the single-DFA and the batch entry points).
//
// The method (arXiv 2410.22764):
//   * Sec. 2: the result is the coarsest partition of all states that refines {F, Q\F} and is
//     stable under delta (language equivalence).
//   * Alg. sortPR (Sec. 3.3): every round gives each state the signature
//         T(s) = (block[s], block[delta(s,0)], ..., block[delta(s,k-1)])
//     and regroups the states by equal signature; rounds repeat until the block count stops
//     changing.  A block may split into many blocks in one round.
//   * Alg. transPR (Sec. 3.4): optionally the alphabet is first extended with the letters
//     a^(2^i), i = 1..floor(log2 n), by pointer doubling; A' has the same state equivalence.
//
// GB300 design (not the paper's Thrust sort):
//   * block ids are LEADER ids: the id of a block is its smallest state.  The block of s in
//     round r+1 is therefore the smallest state with the same signature, which needs no scan;
//     ids are turned into canonical ranks once, at the end (one scan).
//   * a state whose signature equals its leader's keeps its id (this is the test of
//     Alg. naivePR, Sec. 3.2); only the other states are regrouped, through an open-addressing
//     hash table keyed by a 64-bit hash of T(s).  A table hit is accepted only after the FULL
//     signature of the slot's state is compared with T(s), so a hash collision can never merge
//     two groups.  The group id is min(state) by 64-bit atomicMin on the slot.
//   * the count of blocks after a round is (count before) + (table slots claimed), so
//     convergence ("count unchanged") is known on the device after one barrier; there is no
//     host round trip per round.
//   * one launch runs the whole minimization: a persistent cooperative kernel whose CTAs meet at
//     bounded barriers (every wait has a deadline and leaves a status code), or, for DFAs that
//     fit in shared memory, a single CTA with __syncthreads.
//
// Readings of the paper (shared with the CPU oracle): block ids are canonical on output; the
// initial partition is {F, Q\F} without empty parts; a round that leaves the count unchanged
// ends the loop, and so does reaching count == n.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

#include "dfamin.h"

// Internal to the library (the shared object exports only the dfamin_* C functions).
namespace dfamin_dev {

constexpr int kThreads = 256;             // threads per CTA of the one-CTA kernel
#ifndef DFAMIN_TEAM_THREADS
#define DFAMIN_TEAM_THREADS 256           // threads per CTA of the batch and reachability teams
#endif                                    // (the single-DFA team kernel sets its own shape)
#ifndef DFAMIN_TEAM_MIN_CTAS
#define DFAMIN_TEAM_MIN_CTAS 4            // unused by the kernels (kept for builds that set it)
#endif
#ifndef DFAMIN_PREFETCH
#define DFAMIN_PREFETCH 1                 // load the next state's block id and row ahead
#endif
#ifndef DFAMIN_SLOT_CACHE
#define DFAMIN_SLOT_CACHE 128             // per-CTA group-cache entries (rows of <= 8 ints)
#endif
constexpr int kTeamThreads = DFAMIN_TEAM_THREADS;
constexpr int kMaxCtas = 8192;            // capacity of the per-CTA count array
constexpr int64_t kBarrierTimeoutNs = 4000000000ll;        // 4 s per CTA barrier
constexpr int kSmallMaxStates = 8192;     // largest n for the shared-memory kernel
constexpr int kPatMaxK = 8;               // round 1 from acceptance bits for k <= kPatMaxK
constexpr int kPatMax = 1 << (kPatMaxK + 1);

// ------------------------------------------------------------------------------------------
// Device state
// ------------------------------------------------------------------------------------------
struct Ctrl {                      // zeroed by the host before every launch
    unsigned long long bar;        // team barrier: arrivals so far (monotonic)
    unsigned long long claims;     // table slots claimed so far (all rounds)
    int status;                    // first device-detected error
    int min_f_rev;                 // n - (smallest accepting state), 0 if none
    int min_n_rev;                 // n - (smallest rejecting state), 0 if none
    int ncl_letters;               // letters that get closure columns
    int nlead;                     // entries in the global leader list
    int pad0;
    unsigned long long moved;      // states listed as moving so far (all rounds)
    int pad[4];
};

struct Job {
    int32_t n, k;
    const int32_t* __restrict__ delta;   // [n*k] state-major, never written
    const uint32_t* __restrict__ accept; // bitmap
    int64_t acc_off;                     // bit index of state 0 in accept
    int32_t* out_block;                  // [n]
    int32_t* nblocks_out;                // scalar
    int32_t* passes_out;                 // scalar or null
    int32_t* status_out;                 // scalar or null
    int32_t* block;                      // [n] leader ids
    int32_t* cl;                         // closure columns [ncl_letters*(levels-1)][n]
    int32_t* cl_letter;                  // [k] letters with closure columns (compacted)
    int32_t* nonid;                      // [k] 1 if letter is not the identity
    unsigned long long* table;           // [cap] group table: (min state << 32) | representative
                                         // (runtime width) or | old block id (compile-time)
    int32_t* sig;                        // [n * sig_stride] signature rows
    int32_t sig_stride;                  // ints per row, multiple of 4, >= ncols + 1
    int32_t* lst_s;                      // [n] changed states, per-CTA segments
    uint32_t* lst_slot;                  // [n] their table slots (or kCached | cache index)
    uint32_t* lst_rst;                   // [n] slots to empty next round, per-CTA segments
    int32_t* lead;                       // [n] global leader list (append-only)
    uint32_t* lead_slot;                 // [n] table slot of each listed leader's group
    int32_t* stg;                        // [n] per-CTA staging of new leaders
    int32_t* cta_cnt;                    // [kMaxCtas]
    Ctrl* ctrl;
    uint32_t mask;                       // table capacity - 1
    int32_t levels;                      // closure levels (1 = no closure)
    int32_t cl_cols;                     // closure columns the workspace holds (the budget)
    int32_t max_passes;
    uint32_t flags;
    int64_t timeout_ns;
    long long* trace;                    // phase trace or null
    long long trace_cap;                 // records
    int32_t* pat_rev;                    // [kPatMax] round-1 pattern minima (n - state), zeroed
                                         // per launch; null = round 1 by the general path
    int32_t algo;                        // DFAMIN_ALG_SIGNATURE or DFAMIN_ALG_LEADER
    int32_t* naive_new;                  // [n] leader mode: elected new leader per old leader
    int32_t* spl;                        // [n] by leader id: last round in which the block lost
                                         // members (any contents at launch: a stale value can
                                         // only cause extra work)
    int32_t* cln;                        // [n] by leader id: the round in which the block was
                                         // found unable to split (written for every leader in
                                         // every incremental round before it is read)
    // end-to-end calls on page-locked host arrays (else null): round 1 reads every state's row
    // from host memory once and stores the device copy (delta) that later rounds read; the
    // canonical pass writes the labels to host memory
    const int32_t* delta_host;           // [n*k] device-visible alias of the host rows
    int32_t* delta_fill;                 // == delta, writable: the copy round 1 fills
    int32_t* out_host;                   // [n] device-visible alias of the host labels
};

static __device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}


static __device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

static __device__ __forceinline__ void set_status(Ctrl* c, int code) { atomicCAS(&c->status, 0, code); }

// One trace record (written by one thread only).
static __device__ __forceinline__ void trace_mark(const Job& J, bool writer, int pass, int phase)
{
    if (J.trace && writer) {
        const long long i = J.trace[0];
        if (i < J.trace_cap) {
            J.trace[1 + 2 * i] = ((long long)pass << 8) | phase;
            J.trace[2 + 2 * i] = (long long)gtimer();
        }
        J.trace[0] = i + 1;
    }
}

// splitmix64 finalizer (Steele, Lea & Flood 2014); the hash only steers the table probe.
static __device__ __forceinline__ uint64_t fmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static __device__ __forceinline__ uint64_t hash_begin(int leader)
{
    return fmix64((uint64_t)(uint32_t)leader * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull);
}
static __device__ __forceinline__ uint64_t hash_step(uint64_t h, int b)
{
    return fmix64(h + 0x9E3779B97F4A7C15ull + (uint64_t)(uint32_t)b);
}
static __device__ __forceinline__ uint64_t hash_final(uint64_t h, int leader, uint32_t flags)
{
    if (flags & DFAMIN_FLAG_HASH_CONSTANT) return 0;
    if (flags & DFAMIN_FLAG_HASH_BLOCK_ONLY) return hash_begin(leader);
    return h;
}

static __device__ __forceinline__ int is_accepting(const Job& J, int s)
{
    const int64_t b = J.acc_off + s;
    return (int)((__ldg(&J.accept[b >> 5]) >> (b & 31)) & 1u);
}

// Block-id loads.  block[] is written in the kernel (so no non-coherent loads); its random
// gathers are the hot traffic of every round.  With DFAMIN_GATHER_KEEP they carry an L2
// evict-last policy (measured: with the 64-bit group table that is 1.6 % slower on a 10^7-state
// DFA than plain L2 loads, so it is off by default).
#ifndef DFAMIN_GATHER_KEEP
#define DFAMIN_GATHER_KEEP 0
#endif
static __device__ __forceinline__ int ld_blk(const int32_t* p)
{
#if DFAMIN_GATHER_KEEP
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    int v;
    // volatile keeps the load in place relative to barriers; no memory clobber, so independent
    // loads around it (successors, other gathers) can be issued back to back
    asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
#else
    return __ldcg(p);
#endif
}

// Successor of s under signature column c: the k letters, then the closure columns.
static __device__ __forceinline__ int succ_col(const Job& J, int s, int c)
{
    if (c < J.k) return __ldg(&J.delta[(int64_t)s * J.k + c]);
    return __ldcg(&J.cl[(int64_t)(c - J.k) * J.n + s]);
}

// ------------------------------------------------------------------------------------------
// Bounded barrier among the T CTAs of a team.  Monotonic arrival counter: barrier number b is
// passed once the counter reaches b*T.  Every wait has a deadline; on expiry the status word is
// set and every CTA leaves at its next barrier.  Returns false if the team must stop.
// ------------------------------------------------------------------------------------------
struct TeamSync {
    unsigned long long* bar;
    int* status;
    unsigned long long size;
    unsigned long long seq;   // barriers passed (thread 0's copy is the one used)
    int64_t timeout_ns;
};

// The control words a round reads after a barrier, fetched once per CTA (by the thread that
// waited) instead of by every thread: all warps of all CTAs reading one word right after a
// barrier queue thousands of requests at one L2 slice.
struct CtrlSnap {
    unsigned long long claims;
    unsigned long long moved;
    int nlead;
};

static __device__ __forceinline__ bool team_barrier(TeamSync& ts, const Ctrl* src = nullptr,
                                                    CtrlSnap* snap = nullptr)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ts.seq += 1;
        const unsigned long long target = ts.seq * ts.size;
        __threadfence();
        atomicAdd(ts.bar, 1ull);
        int ok = 1;
        if (ld_acquire_u64(ts.bar) < target) {
            const uint64_t t0 = gtimer();
            // tight polling of the counter; the status word and the deadline are checked
            // every 8th poll, and after 256 polls the waiter sleeps between polls
            unsigned it = 0;
            for (;;) {
                if (ld_acquire_u64(ts.bar) >= target) break;
                if ((++it & 7u) == 0u) {
                    if (ld_volatile(ts.status) != 0) { ok = 0; break; }
                    if ((int64_t)(gtimer() - t0) > ts.timeout_ns) {
                        atomicCAS(ts.status, 0, (int)DFAMIN_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (it > 256u) __nanosleep(128);
                }
            }
        }
        __threadfence();
        if (ld_volatile(ts.status) != 0) ok = 0;
        s_ok = ok;
        if (snap) {
            snap->claims = ld_acquire_u64(&src->claims);
            snap->moved = ld_acquire_u64(&src->moved);
            snap->nlead = ld_volatile(&src->nlead);
        }
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive prefix of a 0/1 flag over the CTA's threads; *total receives the CTA sum.
// Must be called by all threads of the CTA.
static __device__ int cta_scan_flag(int flag, int* total)
{
    __shared__ int s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) s_warp[warp] = __popc(ballot);
    __syncthreads();
    if (warp == 0) {
        int v = lane < nwarps ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < nwarps) s_warp[lane] = v;
    }
    __syncthreads();
    const int base = warp ? s_warp[warp - 1] : 0;
    *total = s_warp[nwarps - 1];
    __syncthreads();
    return base + in_warp;
}

// Exclusive prefix of an int over the CTA's threads; *total receives the CTA sum.  Must be
// called by all threads of the CTA.
static __device__ int cta_scan_count(int v, int* total)
{
    __shared__ int s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nwarps) s_warp[lane] = w;
    }
    __syncthreads();
    const int base = warp ? s_warp[warp - 1] : 0;
    *total = s_warp[nwarps - 1];
    __syncthreads();
    return base + x - v;
}

static __device__ int cta_sum(int v)
{
    __shared__ int s_red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    int r = 0;
    for (int w = 0; w < nwarps; ++w) r += s_red[w];
    __syncthreads();
    return r;
}

static __device__ int cta_min(int v)
{
    __shared__ int s_red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    int r = s_red[0];
    for (int w = 1; w < nwarps; ++w) r = min(r, s_red[w]);
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------------------------
// Signature rows.  The signature of s in the current round is T(s) = (block[s],
// block[succ(s,0)], ..., block[succ(s,K-1)]).  The runtime-width rows hold all of it,
// [head, b_0 ..], padded with zeros to a multiple of 4 ints (read and written as int4); the
// compile-time-width rows hold only the successors' ids (the head is known to every reader, see
// RowOf).  A leader writes its row in phase A; a member compares its own signature with its
// leader's row (one sector instead of regathering the leader's successors); a member that
// differs publishes its row before it enters the hash table, so the table can verify equality
// against the row of the state a slot names.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr uint32_t kFail = 0xffffffffu;
// A runtime-width group-table slot holds (smallest member << 32) | representative.  The
// representative is the state that claimed the slot; its row is the one members compare
// against, and it never changes during a round, so only claimers publish rows.  atomicMin on the
// whole word lowers the smallest member and keeps the representative (every member passes the
// same low half).  Compile-time-width slots hold the old block id instead (see insert_row).
constexpr unsigned long long kEmptySlot = ~0ull;

static __device__ __forceinline__ unsigned long long slot_word(int min_state, int rep)
{
    return ((unsigned long long)(uint32_t)min_state << 32) | (uint32_t)rep;
}
static __device__ __forceinline__ int slot_min(unsigned long long w) { return (int)(w >> 32); }
static __device__ __forceinline__ int slot_rep(unsigned long long w) { return (int)(uint32_t)w; }

static __device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

static __device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int SS>
static __device__ __forceinline__ void load_row(const int32_t* sig, int s, int (&row)[SS])
{
    const int4* p = reinterpret_cast<const int4*>(sig + (int64_t)s * SS);
#pragma unroll
    for (int v = 0; v < SS / 4; ++v) {
        const int4 x = __ldcg(p + v);
        row[4 * v] = x.x; row[4 * v + 1] = x.y; row[4 * v + 2] = x.z; row[4 * v + 3] = x.w;
    }
}

template <int SS>
static __device__ __forceinline__ void store_row(int32_t* sig, int s, const int (&row)[SS])
{
    int4* p = reinterpret_cast<int4*>(sig + (int64_t)s * SS);
#pragma unroll
    for (int v = 0; v < SS / 4; ++v)
        __stcg(p + v, make_int4(row[4 * v], row[4 * v + 1], row[4 * v + 2], row[4 * v + 3]));
}

// Successors of s for a compile-time alphabet size KC (state-major delta, streamed once per
// round: evict-first loads).  Vector loads need delta 16-byte aligned (checked on the host).
template <int KC>
static __device__ __forceinline__ void load_succ(const int32_t* __restrict__ delta, int s, int (&r)[KC])
{
    const int32_t* p = delta + (int64_t)s * KC;
    if constexpr (KC % 4 == 0) {
#pragma unroll
        for (int v = 0; v < KC / 4; ++v) {
            const int4 x = __ldcs(reinterpret_cast<const int4*>(p) + v);
            r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
        }
    } else if constexpr (KC % 2 == 0) {
#pragma unroll
        for (int v = 0; v < KC / 2; ++v) {
            const int2 x = __ldcs(reinterpret_cast<const int2*>(p) + v);
            r[2 * v] = x.x; r[2 * v + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < KC; ++c) r[c] = __ldcs(p + c);
    }
}

// Stores the row of s (the device copy filled while reading rows from host memory).
template <int KC>
static __device__ __forceinline__ void store_succ(int32_t* delta, int s, const int (&r)[KC])
{
    int32_t* p = delta + (int64_t)s * KC;
    if constexpr (KC % 4 == 0) {
#pragma unroll
        for (int v = 0; v < KC / 4; ++v)
            reinterpret_cast<int4*>(p)[v] = make_int4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    } else if constexpr (KC % 2 == 0) {
#pragma unroll
        for (int v = 0; v < KC / 2; ++v) reinterpret_cast<int2*>(p)[v] = make_int2(r[2 * v], r[2 * v + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < KC; ++c) p[c] = r[c];
    }
}

// Round 1 reads every state's row (leaders in phase A, the others in phase B), so the range
// check of delta is done there, on rows already in registers, instead of in a separate scan:
// an entry outside [0, n) sets DFAMIN_EINVAL and is never used as an address.
template <int KC>
__device__ __forceinline__ bool row_ok(const Job& J, const int (&r)[KC])
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < KC; ++c) ok &= (unsigned)r[c] < (unsigned)J.n;
    if (!ok) set_status(J.ctrl, DFAMIN_EINVAL);
    return ok;
}

// Row layout of the compile-time-width kernels: the successors' block ids, zero padding to a
// whole number of int4:  [b_0 .. b_{KC-1}, 0 ..], SS = 4 * NB ints (one 16-byte access for
// KC <= 4).  The state's own block id (the head of its signature) is not in the row: a member
// has its leader's head by definition, and movers are grouped under their old block id, which
// the group-table slot holds beside the group's smallest state.
template <int KC>
struct RowOf {
    static constexpr int NB = (KC + 3) / 4;
    static constexpr int SS = 4 * NB;
};

// Letter-masked rounds mark, in a leader's row, the entries that can change this round: bit 31
// of b_a (block ids are below n < 2^31, so the bit is free).  A marked row is read only by the
// round's members; every other reader of a leader's row takes the ids with the bit cleared.
constexpr int kChanged = (int)0x80000000u;
constexpr int kIdBits = 0x7fffffff;


// The first NB int4 of a row: a leader's successor ids (marks cleared).
template <int SS, int NB>
static __device__ __forceinline__ void load_row_prefix(const int32_t* sig, int s, int (&row)[SS])
{
    const int4* p = reinterpret_cast<const int4*>(sig + (int64_t)s * SS);
#pragma unroll
    for (int v = 0; v < NB; ++v) {
        const int4 x = __ldcg(p + v);
        row[4 * v] = x.x & kIdBits; row[4 * v + 1] = x.y & kIdBits;
        row[4 * v + 2] = x.z & kIdBits; row[4 * v + 3] = x.w & kIdBits;
    }
}

// The same, marks kept (letter-masked rounds).
template <int SS, int NB>
static __device__ __forceinline__ void load_row_prefix_marked(const int32_t* sig, int s,
                                                              int (&row)[SS])
{
    const int4* p = reinterpret_cast<const int4*>(sig + (int64_t)s * SS);
#pragma unroll
    for (int v = 0; v < NB; ++v) {
        const int4 x = __ldcg(p + v);
        row[4 * v] = x.x; row[4 * v + 1] = x.y; row[4 * v + 2] = x.z; row[4 * v + 3] = x.w;
    }
}

// The first NB int4 of a row (with SS = 4 * NB, the whole row).
template <int SS, int NB>
static __device__ __forceinline__ void store_row_prefix(int32_t* sig, int s, const int (&row)[SS])
{
    int4* p = reinterpret_cast<int4*>(sig + (int64_t)s * SS);
#pragma unroll
    for (int v = 0; v < NB; ++v)
        __stcg(p + v, make_int4(row[4 * v], row[4 * v + 1], row[4 * v + 2], row[4 * v + 3]));
}

// Publish s's row (the table may point other states at it) before s enters a slot.
template <int SS>
static __device__ __forceinline__ void publish_row(const Job& J, int s, const int (&row)[SS])
{
    store_row<SS>(J.sig, s, row);
    __threadfence();
}

// Compile-time-width group slots hold (smallest member << 32) | head, the head being the old
// block id every member of the group shares.
static __device__ __forceinline__ int slot_head(unsigned long long w) { return (int)(uint32_t)w; }

// Insert s (old block id `head`, successor ids `row`) into the table; returns the slot of s's
// group.  A slot is claimed by CAS from empty; a state whose head and row equal the group's
// lowers the slot's smallest member by atomicMin.  A state publishes its row before it can
// become a slot's smallest member (the claim or the atomicMin), so that the row of the member a
// slot names is always readable: equality is decided on the head and the full row of that
// member, never on the hash.  Other states write nothing.
template <int KC>
static __device__ uint32_t insert_row(const Job& J, int s, int head, uint64_t h,
                                      const int (&row)[RowOf<KC>::SS], int* s_claims,
                                      bool published = false)
{
    constexpr int SS = RowOf<KC>::SS;
    uint32_t idx = (uint32_t)h & J.mask;
    for (uint32_t probe = 0; probe <= J.mask; ++probe) {
        unsigned long long w = ld_acquire_u64(&J.table[idx]);
        if (w == kEmptySlot) {
            if (!published) { publish_row<SS>(J, s, row); published = true; }
            w = atomicCAS(&J.table[idx], kEmptySlot, slot_word(s, head));
            if (w == kEmptySlot) {
                atomicAdd(s_claims, 1);
                return idx;
            }
            __threadfence();   // acquire: the named member's row was published before its atomic
        }
        if (slot_head(w) == head) {
            int tr[SS];
            load_row<SS>(J.sig, slot_min(w), tr);
            bool eq = true;
#pragma unroll
            for (int c = 0; c < KC; ++c) eq &= (tr[c] == row[c]);
            if (eq) {
                if (s < slot_min(w)) {
                    if (!published) { publish_row<SS>(J, s, row); published = true; }
                    atomicMin(&J.table[idx], slot_word(s, head));
                }
                return idx;
            }
        }
        idx = (idx + 1) & J.mask;
    }
    set_status(J.ctrl, DFAMIN_EPROBE);
    return kFail;
}

// Chunks v0 .. v0+3 (16 entries) of the row (head, block[succ(s,0)], ...), with every
// successor load issued before the first gather, and every gather before the first use.
static __device__ __forceinline__ void row_chunk4(const Job& J, int s, int head, int v0, int ncols,
                                           int (&x)[16])
{
    int t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int i = 4 * v0 + j;
        t[j] = (i >= 1 && i <= ncols) ? succ_col(J, s, i - 1) : 0;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int i = 4 * v0 + j;
        if (i >= 1 && i <= ncols && (unsigned)t[j] >= (unsigned)J.n) {
            set_status(J.ctrl, DFAMIN_EINVAL);
            t[j] = 0;
        }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int i = 4 * v0 + j;
        x[j] = i == 0 ? head : (i <= ncols ? ld_blk(&J.block[t[j]]) : 0);
    }
}

// Insert s, whose row is already stored at sig[s], starting at slot idx (runtime width).
static __device__ uint32_t insert_stored_row(const Job& J, int s, uint32_t idx, int nch,
                                             int* s_claims)
{
    const int4* mine = reinterpret_cast<const int4*>(J.sig + (int64_t)s * J.sig_stride);
    for (uint32_t probe = 0; probe <= J.mask; ++probe) {
        unsigned long long w = ld_acquire_u64(&J.table[idx]);
        if (w == kEmptySlot) {
            w = atomicCAS(&J.table[idx], kEmptySlot, slot_word(s, s));
            if (w == kEmptySlot) {
                atomicAdd(s_claims, 1);
                return idx;
            }
            __threadfence();
        }
        const int4* theirs =
            reinterpret_cast<const int4*>(J.sig + (int64_t)slot_rep(w) * J.sig_stride);
        bool eq = true;
        for (int v = 0; v < nch && eq; ++v) {
            const int4 a = __ldcg(mine + v), b = __ldcg(theirs + v);
            eq = a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
        }
        if (eq) {
            if (s < slot_min(w)) atomicMin(&J.table[idx], slot_word(s, slot_rep(w)));
            return idx;
        }
        idx = (idx + 1) & J.mask;
    }
    set_status(J.ctrl, DFAMIN_EPROBE);
    return kFail;
}

// Leader mode (Alg. 2 naivePR): a state that differs from its leader L is elected into the one
// new block split from L this round; the block's new leader is the smallest such state (the
// listing lets any concurrent writer win; the smallest makes runs reproducible).  The list
// entry keeps L, whose election result phase C reads.
__device__ __forceinline__ uint32_t naive_elect(const Job& J, int s, int L)
{
    if ((uint32_t)s < (uint32_t)ld_relaxed_u32((const uint32_t*)&J.naive_new[L]))
        atomicMin(&J.naive_new[L], s);
    return (uint32_t)L;
}

// Counts the leaders (block[s] == s) a warp visits: one shared atomic per warp.  In a round
// that moves nothing these are the final blocks, so the canonical ranks need no extra count.
static __device__ __forceinline__ void count_heads(bool head, int* s_heads)
{
    const unsigned m = __ballot_sync(0xffffffffu, head);
    if ((threadIdx.x & 31u) == 0u && m) atomicAdd(s_heads, __popc(m));
}

// As append_moved, for a loop whose last iteration only some lanes of a warp reach.
static __device__ __forceinline__ void append_moved_partial(const Job& J, int c0, bool moved, int s,
                                                     uint32_t slot, int* s_cnt)
{
    const unsigned act = __activemask();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(act, moved);
    if (m == 0u) return;
    const int first = __ffs(m) - 1;
    int pos0 = 0;
    if ((int)lane == first) pos0 = atomicAdd(s_cnt, __popc(m));
    pos0 = __shfl_sync(act, pos0, first);
    if (moved) {
        const int pos = pos0 + __popc(m & ((1u << lane) - 1u));
        J.lst_s[c0 + pos] = s;
        J.lst_slot[c0 + pos] = slot;
    }
}

// Appends (s, slot) for the lanes with `moved` set: one shared atomic per warp.
static __device__ __forceinline__ void append_moved(const Job& J, int c0, bool moved, int s,
                                             uint32_t slot, int* s_cnt)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, moved);
    if (m == 0u) return;
    const int first = __ffs(m) - 1;
    int pos0 = 0;
    if ((int)lane == first) pos0 = atomicAdd(s_cnt, __popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, first);
    if (moved) {
        const int pos = pos0 + __popc(m & ((1u << lane) - 1u));
        J.lst_s[c0 + pos] = s;
        J.lst_slot[c0 + pos] = slot;
    }
}

// ------------------------------------------------------------------------------------------
// Per-CTA caches for rounds with few blocks.  When the partition has few blocks, most states of
// a CTA fall into a handful of groups, and every probe of the global table would hit the same
// few slots and rows (one L2 slice each).  The CTA then keeps, in shared memory, the groups it
// has already entered (hash, row, global slot) and the rows of leaders it has read.  States are
// visited in increasing order, tile by tile, and a cache entry is filled only by a state that
// went through the global table; a later state that finds its row in the cache is larger than
// that state, so it needs neither the table nor an atomicMin.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kCached = 0x80000000u;  // list slot flag: the low bits index the group cache
#ifndef DFAMIN_CACHE_MAX_BLOCKS
#define DFAMIN_CACHE_MAX_BLOCKS 4096
#endif
constexpr int kCacheMaxBlocks = DFAMIN_CACHE_MAX_BLOCKS;  // rounds starting with at most this many blocks
#ifndef DFAMIN_LEADER_CACHE
#define DFAMIN_LEADER_CACHE 64
#endif
constexpr int kLeaderCache = DFAMIN_LEADER_CACHE;  // leader rows, direct-mapped by leader id

template <int SS>
struct CtaCache {
    static constexpr int kSlots = SS <= 8 ? DFAMIN_SLOT_CACHE : DFAMIN_SLOT_CACHE / 2;
    unsigned long long key[kSlots];
    uint32_t gslot[kSlots];              // kEmpty = entry unused
    int gmin[kSlots];
    int head[kSlots];                    // the group's old block id
    int row[kSlots][SS];
    int lkey[kLeaderCache];
    int lcln[kLeaderCache];              // the leader's clean mark (incremental rounds)
    int lrow[kLeaderCache][SS];
};

template <int KC>
struct CacheOf {
    using type = CtaCache<RowOf<KC>::SS>;
};
template <>
struct CacheOf<0> {
    struct type {
        int unused;
    };
};

template <int SS>
static __device__ void cache_clear(CtaCache<SS>& C)
{
    for (int i = threadIdx.x; i < CtaCache<SS>::kSlots; i += blockDim.x) C.gslot[i] = kEmpty;
    for (int i = threadIdx.x; i < kLeaderCache; i += blockDim.x) C.lkey[i] = -1;
}

template <int KC>
static __device__ void phase_members_cached(const Job& J, int c0, int c1, int* s_claims, int* s_cnt,
                                     CtaCache<RowOf<KC>::SS>& C, int* s_heads, int pass,
                                     bool incr)
{
    constexpr int SS = RowOf<KC>::SS;
    constexpr int kSlots = CtaCache<SS>::kSlots;
    // software pipeline: block[s] and the successor row of the next state are in flight while
    // the current state is processed (in incremental rounds rows are read only when needed)
    int nL = 0, nr[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) nr[c] = 0;
    {
        const int s = c0 + threadIdx.x;
        if (s < c1) {
            nL = ld_blk(&J.block[s]);
            if (!incr) load_succ<KC>(J.delta, s, nr);
        }
    }
    for (int base = c0; base < c1; base += blockDim.x) {
        const int s = base + threadIdx.x;
        int L = nL;
        int r[KC];
#pragma unroll
        for (int c = 0; c < KC; ++c) r[c] = nr[c];
        if (DFAMIN_PREFETCH) {
            if (s + (int)blockDim.x < c1) {
                nL = ld_blk(&J.block[s + blockDim.x]);
                if (!incr) load_succ<KC>(J.delta, s + blockDim.x, nr);
            }
        } else if (s < c1) {
            L = ld_blk(&J.block[s]);
            if (!incr) load_succ<KC>(J.delta, s, r);
        }
        bool moved = false, fill = false, lfill = false, lclean = false;
        uint32_t slot = 0;
        uint64_t h = 0;
        int row[SS], lr[SS];
        count_heads(s < c1 && L == s, s_heads);
        bool visit = s < c1 && L != s;
        if (visit) {
            const int li = L & (kLeaderCache - 1);
            if (C.lkey[li] == L) {
                lclean = incr && C.lcln[li] == pass;
                if (!lclean) {
#pragma unroll
                    for (int c = 0; c < SS; ++c) lr[c] = C.lrow[li][c];
                }
            } else {
                lclean = incr && __ldcg(&J.cln[L]) == pass;
                if (!lclean) load_row_prefix<SS, RowOf<KC>::NB>(J.sig, L, lr);
                lfill = true;
            }
            if (lclean) visit = false;
            else if (incr) load_succ<KC>(J.delta, s, r);
        }
        if (visit && row_ok<KC>(J, r)) {
#pragma unroll
            for (int c = 0; c < KC; ++c) row[c] = ld_blk(&J.block[r[c]]);
#pragma unroll
            for (int c = KC; c < SS; ++c) row[c] = 0;
            bool same = true;
#pragma unroll
            for (int c = 0; c < KC; ++c) same &= (row[c] == lr[c]);
            if (!same) {
                h = hash_begin(L);
#pragma unroll
                for (int c = 0; c < KC; ++c) h = hash_step(h, row[c]);
                h = hash_final(h, L, J.flags);
                const int ci = (int)(h & (uint64_t)(kSlots - 1));
                bool hit = false;
                if (C.gslot[ci] != kEmpty && C.key[ci] == h && C.head[ci] == L) {
                    hit = true;
#pragma unroll
                    for (int c = 0; c < KC; ++c) hit &= (C.row[ci][c] == row[c]);
                }
                if (hit) {
                    slot = kCached | (uint32_t)ci;
                    moved = true;
                } else {
                    slot = insert_row<KC>(J, s, L, h, row, s_claims);
                    moved = fill = slot != kFail;
                }
            }
        }
        append_moved(J, c0, moved, s, slot, s_cnt);
        __syncthreads();                              // lookups of this tile are done
        if (fill) {
            const int ci = (int)(h & (uint64_t)(kSlots - 1));
            if (atomicCAS(&C.gslot[ci], kEmpty, slot) == kEmpty) {
                C.key[ci] = h;
                C.head[ci] = L;
#pragma unroll
                for (int c = 0; c < SS; ++c) C.row[ci][c] = row[c];
            }
        }
        if (lfill) {
            const int li = L & (kLeaderCache - 1);
            if (atomicCAS(&C.lkey[li], -1, L) == -1) {
                C.lcln[li] = lclean ? pass : 0;
                if (!lclean) {
#pragma unroll
                    for (int c = 0; c < SS; ++c) C.lrow[li][c] = lr[c];
                }
            }
        }
        __syncthreads();                              // fills visible to the next tile
    }
}

// ---- incremental rounds.  After a signature round every member of a block B has the same
// row as B's leader (that is how the round grouped them), and the leader's row of that round is
// in sig[] (published by the leader, or stored by it when it moved).  In the next round the
// entry of letter a can change only if the block it names lost members in the round just done
// (spl[] of that block's leader).  So a leader whose stored row names no such block has the same
// row again, and so has every member of its block: the block cannot split this round and its
// members are not visited (cln[leader] = pass tells them).  Only the other blocks are refined
// as usual.  Same partition and same pass count as a full round.
//
// Runtime-width rows ([head, b_0 .. b_{ncols-1}], int4 chunks): is the stored row of leader s
// stale this round?  Writes s's clean mark either way.
static __device__ bool stored_row_dirty(const Job& J, int s, int ncols, int pass)
{
    const int4* row = reinterpret_cast<const int4*>(J.sig + (int64_t)s * J.sig_stride);
    bool dirty = false;
    for (int v = 0; v * 4 <= ncols && !dirty; ++v) {
        const int4 x = __ldcg(row + v);
        const int e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = 4 * v + j;               // entry i is column i - 1
            if (i >= 1 && i <= ncols) {
                const int x = e[j] & kIdBits;
                dirty |= (unsigned)x >= (unsigned)J.n || __ldcg(&J.spl[x]) == pass - 1;
            }
        }
    }
    J.cln[s] = dirty ? 0 : pass;
    return dirty;
}

// ---- phase A: every leader publishes its signature row.  Leaders are kept in a per-CTA list:
// a leader stays a leader (it is the smallest state of its block and stays in its own group),
// and every round adds the smallest states of its new groups.  With `incr` (the previous round
// was a signature round) a leader whose stored row is still valid marks its block clean instead.
template <int KC>
static __device__ void phase_leaders(const Job& J, int rank, int T, int nlead, int ncols,
                                     int pass, bool incr, bool masked)
{
    const int gid = rank * (int)blockDim.x + (int)threadIdx.x, stride = T * (int)blockDim.x;
    if constexpr (KC > 0) {
        constexpr int SS = RowOf<KC>::SS;
        {
            if (masked) {
                // The stored row names the blocks X_a of the last round.  Entry a can change
                // only if X_a lost members in that round (spl[X_a] == pass - 1); the others keep
                // X_a, which is still the id of every state it held.  The row is rewritten with
                // the entries that can change marked: members gather only those.
                // U leaders per thread at a time, every load of a stage issued before any use:
                // the test is a chain of dependent reads (list, old row, split marks, then the
                // successors and the gathers of the marked letters).  A row without marks that
                // needs none is left as it is.
                constexpr int NB = RowOf<KC>::NB;
                constexpr int U = KC <= 2 ? 2 : 1;
                for (int i0 = gid; i0 < nlead; i0 += U * stride) {
                    int sv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int i = i0 + u * stride;
                        sv[u] = i < nlead ? __ldcg(&J.lead[i]) : -1;
                    }
                    int row[U][SS];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (sv[u] >= 0) {
                            load_row_prefix_marked<SS, NB>(J.sig, sv[u], row[u]);
                        } else {
#pragma unroll
                            for (int c = 0; c < SS; ++c) row[u][c] = 0;
                        }
                    }
                    // one leader per thread (wide rows): its successors are read with its row,
                    // before the marks are known, to shorten the chain
                    int r[U][KC];
                    if constexpr (U == 1) {
                        if (sv[0] >= 0) {
                            load_succ<KC>(J.delta, sv[0], r[0]);
                        } else {
#pragma unroll
                            for (int c = 0; c < KC; ++c) r[0][c] = 0;
                        }
                    }
                    unsigned mask[U];
                    bool had[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        mask[u] = 0u;
                        had[u] = false;
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            had[u] |= row[u][c] < 0;
                            const int x = row[u][c] & kIdBits;
                            row[u][c] = x;
                            // an entry outside [0, n) cannot come from this launch's rounds:
                            // the letter is gathered rather than trusted (nothing indexed by it)
                            const bool chg = sv[u] >= 0 && ((unsigned)x >= (unsigned)J.n ||
                                                            __ldcg(&J.spl[x]) == pass - 1);
                            mask[u] |= (chg ? 1u : 0u) << c;
                        }
                    }
                    if constexpr (U > 1) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (mask[u] != 0u) {
                                load_succ<KC>(J.delta, sv[u], r[u]);
                            } else {
#pragma unroll
                                for (int c = 0; c < KC; ++c) r[u][c] = 0;
                            }
                        }
                    }
                    bool put[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        put[u] = sv[u] >= 0 && (mask[u] != 0u || had[u]);
                        if (mask[u] != 0u && !row_ok<KC>(J, r[u])) put[u] = false;
                        if (!put[u]) continue;
#pragma unroll
                        for (int c = 0; c < KC; ++c)
                            if ((mask[u] >> c) & 1u) row[u][c] = ld_blk(&J.block[r[u][c]]) | kChanged;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (!put[u]) continue;
#pragma unroll
                        for (int c = KC; c < SS; ++c) row[u][c] = 0;
                        store_row_prefix<SS, NB>(J.sig, sv[u], row[u]);
                    }
                }
                return;
            }
        }
        if (incr) {
            // U leaders per thread at a time, every load of a stage issued before any use: the
            // test is a chain of dependent reads (list, old row, spl, then delta and gathers)
            constexpr int U = KC <= 2 ? 4 : (KC <= 3 ? 2 : 1);
            constexpr int NB = RowOf<KC>::NB;
            for (int i0 = gid; i0 < nlead; i0 += U * stride) {
                int sv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * stride;
                    sv[u] = i < nlead ? __ldcg(&J.lead[i]) : -1;
                }
                int old[U][4 * NB];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int4* p = reinterpret_cast<const int4*>(J.sig + (int64_t)max(sv[u], 0) * SS);
#pragma unroll
                    for (int v = 0; v < NB; ++v) {
                        const int4 x = sv[u] >= 0 ? __ldcg(p + v) : make_int4(0, 0, 0, 0);
                        old[u][4 * v] = x.x & kIdBits; old[u][4 * v + 1] = x.y & kIdBits;
                        old[u][4 * v + 2] = x.z & kIdBits; old[u][4 * v + 3] = x.w & kIdBits;
                    }
                }
                bool dirty[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    dirty[u] = false;
                    if (sv[u] < 0) continue;
#pragma unroll
                    for (int c = 0; c < KC; ++c)
                        dirty[u] |= (unsigned)old[u][c] >= (unsigned)J.n ||
                                    __ldcg(&J.spl[old[u][c]]) == pass - 1;
                }
                int r[U][KC];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (sv[u] < 0) continue;
                    J.cln[sv[u]] = dirty[u] ? 0 : pass;
                    if (dirty[u]) load_succ<KC>(J.delta, sv[u], r[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (sv[u] < 0 || !dirty[u]) continue;
                    int row[SS];
#pragma unroll
                    for (int c = 0; c < KC; ++c) row[c] = ld_blk(&J.block[r[u][c]]);
#pragma unroll
                    for (int c = KC; c < SS; ++c) row[c] = 0;
                    store_row_prefix<SS, NB>(J.sig, sv[u], row);
                }
            }
            return;
        }
        int ns = 0, nr[KC];
        if (gid < nlead) {
            ns = __ldcg(&J.lead[gid]);
            load_succ<KC>(J.delta, ns, nr);
        }
        for (int i = gid; i < nlead; i += stride) {
            const int s = ns;
            int r[KC];
#pragma unroll
            for (int c = 0; c < KC; ++c) r[c] = nr[c];
            if (i + stride < nlead) {
                ns = __ldcg(&J.lead[i + stride]);
                load_succ<KC>(J.delta, ns, nr);
            }
            if (!row_ok<KC>(J, r)) continue;
            int row[SS];
#pragma unroll
            for (int c = 0; c < KC; ++c) row[c] = ld_blk(&J.block[r[c]]);
#pragma unroll
            for (int c = KC; c < SS; ++c) row[c] = 0;
            store_row_prefix<SS, RowOf<KC>::NB>(J.sig, s, row);
        }
    } else {
        const int nch = (ncols + 4) / 4;
        if ((int64_t)nlead * 4 > (int64_t)J.n) {
            // most states lead: visit the states in order (block[s] == s marks a leader), so a
            // warp reads consecutive entries of every closure column instead of scattered ones
            for (int s = gid; s < J.n; s += stride) {
                if (ld_blk(&J.block[s]) != s) continue;
                if (incr && !stored_row_dirty(J, s, ncols, pass)) continue;
                int4* out = reinterpret_cast<int4*>(J.sig + (int64_t)s * J.sig_stride);
                for (int v0 = 0; v0 < nch; v0 += 4) {
                    int x[16];
                    row_chunk4(J, s, s, v0, ncols, x);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (v0 + u < nch)
                            __stcg(out + v0 + u, make_int4(x[4 * u], x[4 * u + 1], x[4 * u + 2],
                                                           x[4 * u + 3]));
                }
            }
            return;
        }
        for (int i = gid; i < nlead; i += stride) {
            const int s = __ldcg(&J.lead[i]);
            if (incr && !stored_row_dirty(J, s, ncols, pass)) continue;
            int4* out = reinterpret_cast<int4*>(J.sig + (int64_t)s * J.sig_stride);
            for (int v0 = 0; v0 < nch; v0 += 4) {
                int x[16];
                row_chunk4(J, s, s, v0, ncols, x);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (v0 + u < nch)
                        __stcg(out + v0 + u, make_int4(x[4 * u], x[4 * u + 1], x[4 * u + 2],
                                                       x[4 * u + 3]));
            }
        }
    }
}

// A member s of leader L (row r = its successors) compares its signature with L's row; if they
// differ, s is listed to be regrouped (signature mode: its row is stored and its first table
// position returned in *slot) or elected (leader mode).  member_row issues the loads (the
// leader's row and the successors' block ids), member_decide compares and lists; split so that
// the loads of several members can be in flight together.
template <int KC>
static __device__ __forceinline__ void member_row(const Job& J, int L, const int (&r)[KC],
                                                  int (&row)[RowOf<KC>::SS],
                                                  int (&lr)[RowOf<KC>::SS])
{
    constexpr int SS = RowOf<KC>::SS;
    load_row_prefix<SS, RowOf<KC>::NB>(J.sig, L, lr);
#pragma unroll
    for (int c = 0; c < KC; ++c) row[c] = ld_blk(&J.block[r[c]]);
#pragma unroll
    for (int c = KC; c < SS; ++c) row[c] = 0;
}

template <int KC>
static __device__ __forceinline__ bool member_decide(const Job& J, int s, int L,
                                                     const int (&row)[RowOf<KC>::SS],
                                                     const int (&lr)[RowOf<KC>::SS],
                                                     uint32_t* slot)
{
    constexpr int SS = RowOf<KC>::SS;
    bool same = true;
#pragma unroll
    for (int c = 0; c < KC; ++c) same &= (row[c] == lr[c]);
    if (same) return false;
    if (J.algo == DFAMIN_ALG_LEADER) {
        *slot = naive_elect(J, s, L);
        return true;
    }
    // T(s) != T(leader): publish the row and list s with its first probe position; the inserts
    // run afterwards, packed into full warps
    uint64_t h = hash_begin(L);
#pragma unroll
    for (int c = 0; c < KC; ++c) h = hash_step(h, row[c]);
    h = hash_final(h, L, J.flags);
    store_row<SS>(J.sig, s, row);
    *slot = (uint32_t)h & J.mask;
    return true;
}

template <int KC>
static __device__ __forceinline__ bool member_compare(const Job& J, int s, int L, const int (&r)[KC],
                                                      uint32_t* slot)
{
    constexpr int SS = RowOf<KC>::SS;
    int row[SS], lr[SS];
    member_row<KC>(J, L, r, row, lr);
    return member_decide<KC>(J, s, L, row, lr, slot);
}

// ---- phase B of a letter-masked round.  A member s of leader L had L's row in the last round,
// so its entry for an unmarked letter is L's (the block it names kept every state); only the
// marked letters are gathered and compared.  A member whose leader marked nothing keeps its
// block after one row read.  Pipeline: the next state's leader row and the successors of the
// state after it are in flight while the current state's marked letters are gathered.
template <int KC>
static __device__ void members_masked(const Job& J, int c0, int c1, int* s_cnt, int* s_heads)
{
    constexpr int SS = RowOf<KC>::SS;
    constexpr int NB = RowOf<KC>::NB;
    const int bd = (int)blockDim.x;
    int L0 = -1, L1 = -1, r0[KC], r1[KC], lr0[SS];
#pragma unroll
    for (int c = 0; c < KC; ++c) { r0[c] = 0; r1[c] = 0; }
#pragma unroll
    for (int c = 0; c < SS; ++c) lr0[c] = 0;
    {
        const int s = c0 + (int)threadIdx.x;
        if (s < c1) { L0 = ld_blk(&J.block[s]); load_succ<KC>(J.delta, s, r0); }
        if (s + bd < c1) { L1 = ld_blk(&J.block[s + bd]); load_succ<KC>(J.delta, s + bd, r1); }
        if (s < c1 && L0 != s) load_row_prefix_marked<SS, NB>(J.sig, L0, lr0);
    }
    for (int base = c0; base < c1; base += bd) {
        const int s = base + (int)threadIdx.x;
        // issue the next state's leader row and the state after it
        int lr1[SS];
#pragma unroll
        for (int c = 0; c < SS; ++c) lr1[c] = 0;
        if (s + bd < c1 && L1 != s + bd) load_row_prefix_marked<SS, NB>(J.sig, L1, lr1);
        int L2 = -1, r2[KC];
#pragma unroll
        for (int c = 0; c < KC; ++c) r2[c] = 0;
        if (s + 2 * bd < c1) { L2 = ld_blk(&J.block[s + 2 * bd]); load_succ<KC>(J.delta, s + 2 * bd, r2); }

        bool moved = false;
        uint32_t slot = 0;
        count_heads(s < c1 && L0 == s, s_heads);
        bool any = false;
#pragma unroll
        for (int c = 0; c < KC; ++c) any |= lr0[c] < 0;          // bit 31: marked
        if (s < c1 && L0 != s && any && row_ok<KC>(J, r0)) {
            int row[SS];
            bool same = true;
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                const int id = lr0[c] & kIdBits;
                row[c] = lr0[c] < 0 ? ld_blk(&J.block[r0[c]]) : id;
                same &= row[c] == id;
            }
            if (!same) {
#pragma unroll
                for (int c = KC; c < SS; ++c) row[c] = 0;
                uint64_t h = hash_begin(L0);
#pragma unroll
                for (int c = 0; c < KC; ++c) h = hash_step(h, row[c]);
                h = hash_final(h, L0, J.flags);
                store_row<SS>(J.sig, s, row);
                slot = (uint32_t)h & J.mask;
                moved = true;
            }
        }
        append_moved(J, c0, moved, s, slot, s_cnt);
        L0 = L1;
        L1 = L2;
#pragma unroll
        for (int c = 0; c < KC; ++c) { r0[c] = r1[c]; r1[c] = r2[c]; }
#pragma unroll
        for (int c = 0; c < SS; ++c) lr0[c] = lr1[c];
    }
}

// ---- phase B: members compare with their leader; those that differ are regrouped.
// The loop is uniform across the CTA so that appends can be aggregated per warp.
template <int KC>
static __device__ void phase_members(const Job& J, int c0, int c1, int ncols, int* s_claims, int* s_cnt,
                              int* s_heads, int pass, bool incr, bool masked)
{
    if constexpr (KC > 0) {
        constexpr int SS = RowOf<KC>::SS;
        if (masked) {
            members_masked<KC>(J, c0, c1, s_cnt, s_heads);
        } else if (incr) {
            // 1. list the members of blocks that may split (their leader is not marked clean)
            //    in this CTA's segment of stg (states) and lst_rst (leaders).  Pipeline: the
            //    block id of the state after next and the clean mark of the next state's leader
            //    are in flight while the current state is tested.
            __shared__ int s_dcnt;
            if (threadIdx.x == 0) s_dcnt = 0;
            __syncthreads();
            const int bd = (int)blockDim.x;
            int Lc = -1, Cc = 0, Ln = -1;
            {
                const int s0 = c0 + (int)threadIdx.x;
                if (s0 < c1) Lc = ld_blk(&J.block[s0]);
                if (s0 + bd < c1) Ln = ld_blk(&J.block[s0 + bd]);
                if (s0 < c1 && Lc != s0) Cc = __ldcg(&J.cln[Lc]);
            }
            for (int base = c0; base < c1; base += bd) {
                const int s = base + (int)threadIdx.x;
                const int L = Lc, C = Cc;
                Lc = Ln;
                Cc = 0;
                if (s + bd < c1 && Lc != s + bd) Cc = __ldcg(&J.cln[Lc]);
                Ln = s + 2 * bd < c1 ? ld_blk(&J.block[s + 2 * bd]) : -1;
                count_heads(s < c1 && L == s, s_heads);
                const bool visit = s < c1 && L != s && C != pass;
                const unsigned m = __ballot_sync(0xffffffffu, visit);
                if (m) {
                    const unsigned lane = threadIdx.x & 31u;
                    const int first = __ffs(m) - 1;
                    int pos0 = 0;
                    if ((int)lane == first) pos0 = atomicAdd(&s_dcnt, __popc(m));
                    pos0 = __shfl_sync(0xffffffffu, pos0, first);
                    if (visit) {
                        const int pos = c0 + pos0 + __popc(m & ((1u << lane) - 1u));
                        J.stg[pos] = s;
                        J.lst_rst[pos] = (uint32_t)L;
                    }
                }
            }
            __syncthreads();                          // the list (global, this CTA's) is complete
            // 2. the listed members, packed into full warps.  Pipeline: the list entry after next
            //    and the next member's successors are in flight while the current one is tested.
            const int dcnt = s_dcnt;
            int s1 = -1, L1 = 0, s2 = -1, L2 = 0, r1[KC];
            {
                const int i = (int)threadIdx.x;
                if (i < dcnt) { s1 = __ldcg(&J.stg[c0 + i]); L1 = (int)__ldcg(&J.lst_rst[c0 + i]); }
                if (i + bd < dcnt) {
                    s2 = __ldcg(&J.stg[c0 + i + bd]);
                    L2 = (int)__ldcg(&J.lst_rst[c0 + i + bd]);
                }
                if (s1 >= 0) load_succ<KC>(J.delta, s1, r1);
            }
            for (int i = (int)threadIdx.x; i < dcnt; i += bd) {
                const int sv = s1, Lv = L1;
                int r[KC];
#pragma unroll
                for (int c = 0; c < KC; ++c) r[c] = r1[c];
                s1 = s2;
                L1 = L2;
                if (s1 >= 0) load_succ<KC>(J.delta, s1, r1);
                s2 = -1;
                if (i + 2 * bd < dcnt) {
                    s2 = __ldcg(&J.stg[c0 + i + 2 * bd]);
                    L2 = (int)__ldcg(&J.lst_rst[c0 + i + 2 * bd]);
                }
                uint32_t slot = 0;
                const bool moved = row_ok<KC>(J, r) && member_compare<KC>(J, sv, Lv, r, &slot);
                // every lane of the warp is in the loop while any is: the loop bound is uniform
                // per warp only up to the last iteration, so the append is warp-synchronous on
                // the lanes still in it
                append_moved_partial(J, c0, moved, sv, slot, s_cnt);
            }
        } else {
        int nL = 0, nr[KC];
        {
            const int s = c0 + threadIdx.x;
            if (s < c1) { nL = ld_blk(&J.block[s]); load_succ<KC>(J.delta, s, nr); }
        }
        for (int base = c0; base < c1; base += blockDim.x) {
            const int s = base + threadIdx.x;
            int L = nL;
            int r[KC];
#pragma unroll
            for (int c = 0; c < KC; ++c) r[c] = nr[c];
            if (DFAMIN_PREFETCH) {
                if (s + (int)blockDim.x < c1) {
                    nL = ld_blk(&J.block[s + blockDim.x]);
                    load_succ<KC>(J.delta, s + blockDim.x, nr);
                }
            } else if (s < c1) {
                L = ld_blk(&J.block[s]);
                load_succ<KC>(J.delta, s, r);
            }
            bool moved = false;
            uint32_t slot = 0;
            count_heads(s < c1 && L == s, s_heads);
            if (s < c1 && L != s && row_ok<KC>(J, r)) moved = member_compare<KC>(J, s, L, r, &slot);
            append_moved(J, c0, moved, s, slot, s_cnt);
        }
        }
        if (J.algo != DFAMIN_ALG_LEADER) {
            // ---- regroup the listed states: every lane of a warp has an insert to do
            // Ordering: every writer fences its own row stores (they are performed in L2, the
            // point of coherence) before the CTA barrier, and a slot is claimed only after the
            // barrier; a reader that sees the claim (ld.acquire) reads the row from L2 (ld.cg),
            // so it never sees an older row.
            __threadfence();                          // each thread's rows visible device-wide
            __syncthreads();                          // ... before any lane claims a slot
            const int cnt = *s_cnt;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int s = __ldcg(&J.lst_s[c0 + i]);
                const uint32_t idx = __ldcg(&J.lst_slot[c0 + i]);
                int row[SS];
                load_row<SS>(J.sig, s, row);
                const int head = ld_blk(&J.block[s]);   // s's old block (rewritten in phase C)
                const uint32_t slot = insert_row<KC>(J, s, head, (uint64_t)idx, row, s_claims, true);
                J.lst_slot[c0 + i] = slot;
            }
        }
    } else {
        const int nch = (ncols + 4) / 4;
        const bool defer = J.algo != DFAMIN_ALG_LEADER;
        for (int base = c0; base < c1; base += blockDim.x) {
            const int s = base + threadIdx.x;
            bool moved = false;
            uint32_t slot = 0;
            int L = -1;
            if (s < c1) L = ld_blk(&J.block[s]);
            count_heads(s < c1 && L == s, s_heads);
            if (s < c1) {
                if (L != s && (!incr || __ldcg(&J.cln[L]) != pass)) {
                    const int4* lrow =
                        reinterpret_cast<const int4*>(J.sig + (int64_t)L * J.sig_stride);
                    int4* mine = reinterpret_cast<int4*>(J.sig + (int64_t)s * J.sig_stride);
                    bool same = true;
                    int stored = 0;                   // leading chunks of the row written
                    uint64_t h = hash_begin(L);
                    for (int v0 = 0; v0 < nch; v0 += 4) {
                        int4 l[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (v0 + u < nch) l[u] = __ldcg(lrow + v0 + u);
                        int x[16];
                        row_chunk4(J, s, L, v0, ncols, x);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int i = 4 * v0 + j;
                            if (i >= 1 && i <= ncols) h = hash_step(h, x[j]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (v0 + u >= nch) break;
                            const int* y = x + 4 * u;
                            same = same && l[u].x == y[0] && l[u].y == y[1] && l[u].z == y[2] &&
                                   l[u].w == y[3];
                        }
                        // a regrouping state writes its row once, so that its inserts compare
                        // stored rows; the chunks it shares with its leader are copied
                        if (defer && !same) {
                            for (int v = stored; v < v0; ++v) __stcg(mine + v, __ldcg(lrow + v));
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (v0 + u < nch)
                                    __stcg(mine + v0 + u, make_int4(x[4 * u], x[4 * u + 1],
                                                                    x[4 * u + 2], x[4 * u + 3]));
                            stored = min(v0 + 4, nch);
                        }
                    }
                    if (!same && J.algo == DFAMIN_ALG_LEADER) {
                        slot = naive_elect(J, s, L);
                        moved = true;
                    } else if (!same) {
                        h = hash_final(h, L, J.flags);
                        slot = (uint32_t)h & J.mask;
                        moved = true;
                    }
                }
            }
            append_moved(J, c0, moved, s, slot, s_cnt);
        }
        if (defer) {
            // ---- regroup the listed states, packed into full warps (rows already stored)
            __threadfence();
            __syncthreads();
            const int cnt = *s_cnt;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int s = __ldcg(&J.lst_s[c0 + i]);
                const uint32_t idx = __ldcg(&J.lst_slot[c0 + i]);
                J.lst_slot[c0 + i] = insert_stored_row(J, s, idx, nch, s_claims);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Team kernel body: one DFA refined by T co-resident CTAs; CTA `rank` owns states [c0, c1).
// Per round: A (reset last round's slots, leaders publish rows) | B (members) | C (moves).
// ------------------------------------------------------------------------------------------
static __device__ void write_outputs(const Job& J, int nblocks, int passes)
{
    const int st = ld_volatile(&J.ctrl->status);
    *J.nblocks_out = st ? -st : nblocks;
    if (J.passes_out) *J.passes_out = passes;
    if (J.status_out) *J.status_out = st;
}

// Stages (new leader, its group's slot) for the flagged lanes in this CTA's segment of the
// staging lists (one shared atomic per warp).
static __device__ __forceinline__ void append_pair(const Job& J, int c0, int* cnt, bool flag, int s,
                                            uint32_t slot)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (m == 0u) return;
    const int first = __ffs(m) - 1;
    int pos0 = 0;
    if ((int)lane == first) pos0 = atomicAdd(cnt, __popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, first);
    if (flag) {
        const int pos = c0 + pos0 + __popc(m & ((1u << lane) - 1u));
        J.stg[pos] = s;
        J.lst_rst[pos] = slot;
    }
}

// ------------------------------------------------------------------------------------------
// Closure columns of Alg. transPR (Sec. 3.4), level-major: level i of every letter that is
// still changing is stored in consecutive columns after those of level i-1.  Level i of letter a
// is level i-1 applied twice.  When level i of a letter equals its level i-1 for every state,
// every later level equals it too, so the letter gets no further levels; its level-i column (a
// copy of level i-1) stays, since a repeated column changes no signature comparison.  With
// DFAMIN_FLAG_KEEP_IDENTITY, or with more than kClSatLetters closed letters, every level of
// every letter is built.  Letters are cl_letter[0..ncl); nonid[a] holds 1 (a is not the
// identity) and then i+1 once level i of a is seen to differ from level i-1.
// Team form (ts != nullptr): this CTA builds states [c0, c1) and every level ends with a team
// barrier.  One-CTA form: states [0, n), __syncthreads.  Returns the number of closure columns,
// or -1 when the team must stop.
// ------------------------------------------------------------------------------------------
constexpr int kClSatLetters = 128;

static __device__ int closure_build(const Job& J, int c0, int c1, int ncl, TeamSync* ts, bool tw)
{
    __shared__ int s_act[kClSatLetters], s_src[kClSatLetters];
    __shared__ int s_na;
    const int n = J.n, k = J.k, lv = J.levels - 1;
    const bool sat = !(J.flags & DFAMIN_FLAG_KEEP_IDENTITY) && ncl <= kClSatLetters;
    if (sat) {
        for (int r = threadIdx.x; r < ncl; r += blockDim.x) {
            s_act[r] = __ldcg(&J.cl_letter[r]);
            s_src[r] = -1;
        }
    }
    __syncthreads();
    int na = ncl, ncol = 0;
    for (int i = 1; i <= lv && na > 0; ++i) {
        // column budget: a level that does not fit whole is built for its first letters only,
        // and no level follows it (missing columns only cost rounds: every subset of the closed
        // alphabet has the same state equivalence)
        const int nb = min(na, J.cl_cols - ncol);
        if (nb <= 0) break;
        const bool truncated = nb < na;
        for (int r = 0; r < nb; ++r) {
            const int a = sat ? s_act[r] : __ldcg(&J.cl_letter[r]);
            const int src = sat ? s_src[r] : (i == 1 ? -1 : ncol - na + r);
            const int32_t* prev = J.cl + (int64_t)src * n;
            int32_t* cur = J.cl + (int64_t)(ncol + r) * n;
            bool changed = false;
            for (int q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
                int t1, t;
                if (src < 0) {
                    t1 = __ldg(&J.delta[(int64_t)q * k + a]);
                    t = __ldg(&J.delta[(int64_t)t1 * k + a]);
                } else {
                    t1 = __ldcg(&prev[q]);
                    t = __ldcg(&prev[t1]);
                }
                cur[q] = t;
                changed |= t != t1;
            }
            if (sat) {
                if (__syncthreads_or(changed) && threadIdx.x == 0) J.nonid[a] = i + 1;
            }
        }
        ncol += nb;
        if (ts) {
            if (!team_barrier(*ts)) return -1;
        } else {
            __syncthreads();
        }
        trace_mark(J, tw, i, 3);
        if (sat) {
            if (threadIdx.x == 0) {
                int m = 0;
                for (int r = 0; r < nb; ++r) {
                    const int a = s_act[r];
                    if (ld_volatile(&J.nonid[a]) == i + 1) {
                        s_act[m] = a;
                        s_src[m] = ncol - nb + r;
                        ++m;
                    }
                }
                s_na = m;
            }
            __syncthreads();
            // no letter changed at level i: the whole level repeats level i-1, drop it
            if (s_na == 0) ncol -= nb;
            na = s_na;
            __syncthreads();
        }
        if (truncated) break;
    }
    return ncol;
}

template <int KC>
static __device__ void team_minimize(const Job& J, int rank, int T, TeamSync& ts)
{
    __shared__ int s_claims;
    __shared__ int s_cnt;
    __shared__ int s_rst;
    __shared__ int s_base;
    __shared__ int s_heads;
    bool heads_valid = false;                          // cta_cnt holds this CTA's leader count
    const int n = J.n, k = J.k;
    // chunks are multiples of 32 states so that every CTA's rows start 16-byte aligned
    const int chunk = ((n + T - 1) / T + 31) / 32 * 32;
    const int c0 = min(n, rank * chunk), c1 = min(n, c0 + chunk);
    const bool closure = J.levels > 1;
    const bool elide = !(J.flags & DFAMIN_FLAG_KEEP_IDENTITY);
    int passes = 0;
    bool round1_done = false, round2_done = false;
    int round1_count0 = 0, round1_count1 = 0, round1_count2 = 0;
    const bool tw = rank == 0 && threadIdx.x == 0;     // trace writer
    if (threadIdx.x == 0) { s_claims = 0; s_cnt = 0; s_rst = 0; }
    trace_mark(J, tw, 0, 0);

    // ---- round 1 from the acceptance bits.  In P0 = {F, Q\F} a state's signature is fixed by
    //      the acceptance of the state and of its k successors, so round 1 groups the states by
    //      that (k+1)-bit pattern (exact: the pattern is the signature written in bits), and a
    //      group's id is its smallest state (per-CTA minima in shared memory, then one atomic per
    //      CTA and pattern).  It replaces phases V and I and the general round 1, with the same
    //      partition and pass count.
    if constexpr (KC > 0 && KC <= kPatMaxK) {
        if (J.pat_rev && !closure && J.algo == DFAMIN_ALG_SIGNATURE) {
            constexpr int NP = 1 << (KC + 1);
            using PatT = typename std::conditional<(KC <= 7), uint8_t, int32_t>::type;
            __shared__ int s_pat[NP];
            for (int i = threadIdx.x; i < NP; i += blockDim.x) s_pat[i] = 0x7fffffff;
            __syncthreads();
            bool bad = false;
            // the next state's row is in flight while this one's successors are looked up.
            // From host memory (end-to-end calls) every row is read once here and stored to the
            // device copy that the later rounds read.
            const int32_t* rows = J.delta_host ? J.delta_host : J.delta;
            int nr[KC];
            if (c0 + (int)threadIdx.x < c1) load_succ<KC>(rows, c0 + (int)threadIdx.x, nr);
            for (int q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
                int r[KC];
#pragma unroll
                for (int c = 0; c < KC; ++c) r[c] = nr[c];
                if (q + (int)blockDim.x < c1) load_succ<KC>(rows, q + (int)blockDim.x, nr);
                if (J.delta_host) store_succ<KC>(J.delta_fill, q, r);
                int pat = is_accepting(J, q) ? 1 : 0;
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                    if ((unsigned)r[c] >= (unsigned)n) bad = true;
                    else pat |= (is_accepting(J, r[c]) ? 1 : 0) << (c + 1);
                }
                // the pattern, until the ids are known (one byte a state for k <= 7: the dense
                // round 2 gathers it from an array a quarter the size)
                reinterpret_cast<PatT*>(J.naive_new)[q] = (PatT)pat;
                if (q < s_pat[pat]) atomicMin(&s_pat[pat], q);
            }
            if (bad) set_status(J.ctrl, DFAMIN_EINVAL);
            const uint64_t cap = (uint64_t)J.mask + 1;
            const uint64_t per = (cap + T - 1) / T;
            const uint64_t t0 = min(cap, per * rank), t1 = min(cap, t0 + per);
            for (uint64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) J.table[i] = kEmptySlot;
            __syncthreads();
            for (int i = threadIdx.x; i < NP; i += blockDim.x)
                if (s_pat[i] != 0x7fffffff) atomicMax(&J.pat_rev[i], n - s_pat[i]);
            if (!team_barrier(ts)) goto done;
            trace_mark(J, tw, 1, 5);
            for (int i = threadIdx.x; i < NP; i += blockDim.x) s_pat[i] = ld_volatile(&J.pat_rev[i]);
            __syncthreads();
            int c1cnt = 0, has_f = 0, has_n = 0;
            for (int i = 0; i < NP; ++i) {
                if (s_pat[i] > 0) {
                    ++c1cnt;
                    if (i & 1) has_f = 1; else has_n = 1;
                }
            }
            round1_count0 = has_f + has_n;
            round1_count1 = c1cnt;
            // round 2 by dense codes (below) needs only the patterns: then round 1's ids and
            // leader list, which it would overwrite, are not written
            constexpr int PB = KC + 1;
            constexpr int CB = 1 + KC * PB;           // bits of a round-2 code (below)
            bool dense_next = false;
            if constexpr (CB <= 26) {
                const uint64_t words = 2ull * ((uint64_t)J.mask + 1);
                dense_next = round1_count1 != round1_count0 && round1_count1 < n &&
                             J.max_passes >= 2 && (1ull << CB) <= words;
            }
            if (!dense_next) {
                for (int q = c0 + threadIdx.x; q < c1; q += blockDim.x)
                    J.block[q] = n - s_pat[reinterpret_cast<const PatT*>(J.naive_new)[q]];
                if (rank == 0 && threadIdx.x == 0) {
                    int m = 0;
                    for (int i = 0; i < NP; ++i)
                        if (s_pat[i] > 0) J.lead[m++] = n - s_pat[i];
                    J.ctrl->nlead = m;
                }
                if (!team_barrier(ts)) goto done;
                trace_mark(J, tw, 1, 6);
            }
            round1_done = true;

            // ---- round 2 by dense codes.  After round 1 a block is a (k+1)-bit pattern, so a
            //      state's round-2 signature is exactly the patterns of the state and of its
            //      successors.  The state's own pattern repeats the successors' acceptance bits,
            //      which their patterns hold too, so the signature is exactly the code of the
            //      state's acceptance and its successors' patterns: 1 + k(k+1) bits (21 for
            //      k = 4).  For k <= 4 the code indexes a direct table (the group table's memory
            //      seen as 32-bit words, all ones = empty; 8 MB for k = 4, so that the groups'
            //      words stay in L2): one atomicMin per state gives every group its smallest
            //      state, with no hashing and no row comparison.  Same partition and pass count
            //      as the general round.
            if constexpr (CB <= 26) {
                if (dense_next) {
                    uint32_t* dtab = reinterpret_cast<uint32_t*>(J.table);
                    const PatT* pidx = reinterpret_cast<const PatT*>(J.naive_new);
                    if (threadIdx.x == 0) s_claims = 0;
                    __syncthreads();
                    int mine = 0;
                    // two states per thread per step: their gathers and atomics overlap; the
                    // rows of the next step's states are in flight meanwhile
                    const int bd = (int)blockDim.x;
                    int nr[2][KC];
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if (c0 + (int)threadIdx.x + u * bd < c1)
                            load_succ<KC>(J.delta, c0 + (int)threadIdx.x + u * bd, nr[u]);
                    for (int q0 = c0 + threadIdx.x; q0 < c1; q0 += 2 * blockDim.x) {
                        uint32_t code[2];
                        int qv[2] = {q0, q0 + (int)blockDim.x};
                        int rr[2][KC];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
#pragma unroll
                            for (int c = 0; c < KC; ++c) rr[u][c] = nr[u][c];
                            if (qv[u] + 2 * bd < c1) load_succ<KC>(J.delta, qv[u] + 2 * bd, nr[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            code[u] = 0;
                            if (qv[u] >= c1) continue;
                            const int (&r)[KC] = rr[u];
                            code[u] = (uint32_t)__ldcs(&pidx[qv[u]]) & 1u;   // acceptance of q
#pragma unroll
                            for (int c = 0; c < KC; ++c)
                                code[u] |= (uint32_t)__ldcg(&pidx[r[c]]) << (1 + c * PB);
                        }
                        uint32_t old[2] = {0u, 0u};
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            if (qv[u] >= c1) continue;
                            J.lst_slot[qv[u]] = code[u];
                            old[u] = atomicMin(&dtab[code[u]], (uint32_t)qv[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) mine += qv[u] < c1 && old[u] == 0xffffffffu;
                    }
                    mine = cta_sum(mine);
                    if (threadIdx.x == 0) {
                        if (mine) atomicAdd(&J.ctrl->claims, (unsigned long long)mine);
                        if (rank == 0) J.ctrl->nlead = 0;    // the list is rebuilt below
                    }
                    if (!team_barrier(ts)) goto done;
                    trace_mark(J, tw, 2, 5);
                    round1_count2 = (int)ld_acquire_u64(&J.ctrl->claims);
                    // every group's smallest state leads it and lists its table word for reset
                    if (threadIdx.x == 0) s_rst = 0;
                    __syncthreads();
                    // four states per thread per step; the next step's codes are in flight
                    uint32_t ncv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = c0 + u * (int)blockDim.x + (int)threadIdx.x;
                        ncv[u] = q < c1 ? __ldcs(&J.lst_slot[q]) : 0u;
                    }
                    for (int b = c0; b < c1; b += 4 * (int)blockDim.x) {
                        int qv[4], mv[4];
                        uint32_t cv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            qv[u] = b + u * (int)blockDim.x + (int)threadIdx.x;
                            cv[u] = ncv[u];
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            mv[u] = qv[u] < c1 ? (int)__ldcg(&dtab[cv[u]]) : -1;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = qv[u] + 4 * (int)blockDim.x;
                            ncv[u] = q < c1 ? __ldcs(&J.lst_slot[q]) : 0u;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (qv[u] < c1) J.block[qv[u]] = mv[u];
                            append_pair(J, c0, &s_rst, qv[u] < c1 && mv[u] == qv[u], qv[u],
                                        cv[u] >> 1);
                        }
                    }
                    __syncthreads();
                    const int nnew = s_rst;
                    if (threadIdx.x == 0) s_base = nnew ? atomicAdd(&J.ctrl->nlead, nnew) : 0;
                    __syncthreads();
                    for (int i = threadIdx.x; i < nnew; i += blockDim.x) {
                        J.lead[s_base + i] = J.stg[c0 + i];
                        J.lead_slot[s_base + i] = J.lst_rst[c0 + i];
                    }
                    if (!team_barrier(ts)) goto done;
                    trace_mark(J, tw, 2, 6);
                    round2_done = true;
                }
            }
        }
    }
    if (!round1_done) {
        // ---- phase V: validate delta rows, find the two initial leaders, mark identity letters,
        //      empty this CTA's slice of the hash table
        {
            bool bad = false;
            const int64_t r0 = (int64_t)c0 * k, r1 = (int64_t)c1 * k;
            if (!closure && n > 2) {
                // validated in round 1 (row_ok / row_chunk)
            } else if (!closure && ((uintptr_t)J.delta & 15u) == 0) {
                const int64_t v0 = r0 / 4, v1 = r1 / 4;   // r0 is a multiple of 4 (chunk % 32 == 0)
                const int4* d4 = reinterpret_cast<const int4*>(J.delta);
                for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
                    const int4 v = __ldcs(d4 + i);
                    bad |= ((unsigned)v.x >= (unsigned)n) | ((unsigned)v.y >= (unsigned)n) |
                           ((unsigned)v.z >= (unsigned)n) | ((unsigned)v.w >= (unsigned)n);
                }
                for (int64_t i = v1 * 4 + threadIdx.x; i < r1; i += blockDim.x)
                    bad |= (unsigned)__ldcs(&J.delta[i]) >= (unsigned)n;
            } else {
                for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
                    const int v = __ldcs(&J.delta[i]);
                    if ((unsigned)v >= (unsigned)n) bad = true;
                    if (closure && v != (int)(i / k)) J.nonid[i % k] = 1;
                }
            }
            if (bad) set_status(J.ctrl, DFAMIN_EINVAL);
            int mf = 0x7fffffff, mn = 0x7fffffff;
            for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
                if (is_accepting(J, s)) mf = min(mf, s); else mn = min(mn, s);
            }
            mf = cta_min(mf);
            mn = cta_min(mn);
            if (threadIdx.x == 0) {
                if (mf != 0x7fffffff) atomicMax(&J.ctrl->min_f_rev, n - mf);
                if (mn != 0x7fffffff) atomicMax(&J.ctrl->min_n_rev, n - mn);
            }
            const uint64_t cap = (uint64_t)J.mask + 1;
            const uint64_t per = (cap + T - 1) / T;
            const uint64_t t0 = min(cap, per * rank), t1 = min(cap, t0 + per);
            for (uint64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) J.table[i] = kEmptySlot;
            if (J.algo == DFAMIN_ALG_LEADER)
                for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x) J.naive_new[i] = 0x7fffffff;
        }
        if (!team_barrier(ts)) goto done;
        trace_mark(J, tw, 0, 1);

        // ---- phase I: initial partition P0 = {F, Q\F} as leader ids
        {
            const int rf = ld_volatile(&J.ctrl->min_f_rev), rn = ld_volatile(&J.ctrl->min_n_rev);
            const int lf = n - rf, ln = n - rn;
            for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x)
                J.block[s] = is_accepting(J, s) ? lf : ln;
            if (rank == 0 && threadIdx.x == 0) {
                int m = 0;
                if (rf > 0) J.lead[m++] = lf;
                if (rn > 0) J.lead[m++] = ln;
                J.ctrl->nlead = m;
            }
            if (closure && rank == 0 && threadIdx.x == 0) {
                int m = 0;
                for (int a = 0; a < k; ++a)
                    if (!elide || ld_volatile(&J.nonid[a])) J.cl_letter[m++] = a;
                J.ctrl->ncl_letters = m;
            }
        }
        if (!team_barrier(ts)) goto done;
        trace_mark(J, tw, 0, 2);
    }

    {
        int count = round2_done   ? round1_count2
                    : round1_done ? round1_count1
                                  : (ld_volatile(&J.ctrl->min_f_rev) > 0) +
                                        (ld_volatile(&J.ctrl->min_n_rev) > 0);
        // a discrete P0 (n <= 2) needs no round at all, as in the general path
        if (round1_done) passes = round1_count0 < n ? 1 : 0;
        if (round2_done) passes = 2;
        int ncl_cols = 0;
        if constexpr (KC == 0) {
            // ---- closure levels (Alg. transPR)
            if (closure) {
                ncl_cols = closure_build(J, c0, c1, ld_volatile(&J.ctrl->ncl_letters), &ts, tw);
                if (ncl_cols < 0) goto done;
            }
        }
        const int ncols = k + ncl_cols;
        // ---- runtime-width round 1 by acceptance keys.  In P0 a signature is exactly the
        //      acceptance of the state and of its ncols successors; with ncols < 32 that is a
        //      32-bit key, stored in the table slot beside the group's smallest state (slot =
        //      (min << 32) | key), so the round publishes and compares no rows.
        bool keys_done = false;
        int keys_count0 = count;
        if constexpr (KC == 0) {
            if (!round1_done && J.algo == DFAMIN_ALG_SIGNATURE && ncols < 32 && count < n) {
                int mine = 0;
                for (int q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
                    uint32_t key = is_accepting(J, q) ? 1u : 0u;
                    for (int b = 0; b < ncols; b += 16) {
                        int t[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) t[j] = b + j < ncols ? succ_col(J, q, b + j) : 0;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (b + j >= ncols) continue;
                            if ((unsigned)t[j] >= (unsigned)n) set_status(J.ctrl, DFAMIN_EINVAL);
                            else key |= (is_accepting(J, t[j]) ? 1u : 0u) << (b + j + 1);
                        }
                    }
                    uint64_t hk = (uint64_t)key * 0x9E3779B97F4A7C15ull;
                    hk ^= hk >> 29;
                    uint32_t idx = (uint32_t)hk & J.mask;
                    uint32_t probe = 0;
                    for (; probe <= J.mask; ++probe) {
                        unsigned long long w = ld_acquire_u64(&J.table[idx]);
                        if (w == kEmptySlot) {
                            w = atomicCAS(&J.table[idx], kEmptySlot, slot_word(q, (int)key));
                            if (w == kEmptySlot) { ++mine; break; }
                        }
                        if ((uint32_t)w == key) {
                            if (q < slot_min(w)) atomicMin(&J.table[idx], slot_word(q, (int)key));
                            break;
                        }
                        idx = (idx + 1) & J.mask;
                    }
                    if (probe > J.mask) set_status(J.ctrl, DFAMIN_EPROBE);
                    J.lst_slot[q] = idx;
                }
                mine = cta_sum(mine);
                if (threadIdx.x == 0) {
                    if (mine) atomicAdd(&J.ctrl->claims, (unsigned long long)mine);
                    if (rank == 0) J.ctrl->nlead = 0;    // the list is rebuilt below
                }
                if (!team_barrier(ts)) goto done;
                trace_mark(J, tw, 1, 5);
                // every group's smallest state leads it and lists its slot for reset
                if (threadIdx.x == 0) s_rst = 0;
                __syncthreads();
                for (int b = c0; b < c1; b += blockDim.x) {
                    const int q = b + (int)threadIdx.x;
                    bool lead = false;
                    uint32_t slot = 0;
                    if (q < c1) {
                        slot = __ldcs(&J.lst_slot[q]);
                        const int m = slot_min(__ldcg(&J.table[slot]));
                        J.block[q] = m;
                        lead = m == q;
                    }
                    append_pair(J, c0, &s_rst, lead, q, slot);
                }
                __syncthreads();
                const int nnew = s_rst;
                if (threadIdx.x == 0) s_base = nnew ? atomicAdd(&J.ctrl->nlead, nnew) : 0;
                __syncthreads();
                for (int i = threadIdx.x; i < nnew; i += blockDim.x) {
                    J.lead[s_base + i] = J.stg[c0 + i];
                    J.lead_slot[s_base + i] = J.lst_rst[c0 + i];
                }
                if (!team_barrier(ts)) goto done;
                trace_mark(J, tw, 1, 6);
                count = (int)ld_acquire_u64(&J.ctrl->claims);
                passes = 1;
                keys_done = true;
            }
        }
        const int max_passes = J.max_passes;
        unsigned long long claims_seen = round2_done ? (unsigned long long)round1_count2
                                         : keys_done ? (unsigned long long)count
                                                     : 0ull;
        // leaders of the first rounds own no group slot, except after the dense round 2 or
        // the key round, whose every leader lists the slot it used
        int lead_reset_from = (round2_done || keys_done) ? 0 : ld_volatile(&J.ctrl->nlead);
        const bool leader_mode = J.algo == DFAMIN_ALG_LEADER;
        // signature rounds stop early once every block is a singleton; Alg. 2 runs until a
        // round changes nothing
        // round 1 (or 2) done above and nothing split: stable
        const bool stable1 = (round1_done && round1_count1 == round1_count0) ||
                             (round2_done && round1_count2 == round1_count1) ||
                             (keys_done && count == keys_count0);
        // rows of the last round are in sig[] for every leader once a signature round has run
        // (not after the pattern, dense-code or key rounds)
        bool have_rows = false;
        unsigned long long moved_seen = 0, moved_last = 0;
        __shared__ CtrlSnap s_snap;
        int nlead_cur = ld_volatile(&J.ctrl->nlead);      // leaders listed for the next round
        while (!stable1 && (leader_mode || count < n)) {
            if (passes >= max_passes) {
                set_status(J.ctrl, DFAMIN_ENOCONVERGE);
                break;
            }
            ++passes;
            // an incremental round pays off when few blocks can split: the states that moved in
            // the last round mark their old blocks, and a block is revisited when its row names
            // one of them, so with M movers and ncols columns about ncols * 2M / n of the blocks
            // are revisited.  Below a quarter of that bound the round is incremental.
            // a letter-masked round (rows of 8 ints or with room for the mask) reads one leader
            // row per member and gathers only the letters whose block split; it replaces the
            // incremental round and, while members outnumber leaders, the full one (a leader
            // pays one row read and k split marks more, a member saves the unmarked gathers).
            // With few blocks the per-CTA caches serve the leader rows instead.
            const int nlead_round = nlead_cur;
            // (compile-time widths only: for the runtime width the extra code cost registers and
            // the marks saved nothing on the bit-splitters and the batches' random DFAs)
            const bool masked =
                KC > 0 && have_rows && !leader_mode &&
                !(J.flags & (DFAMIN_FLAG_FULL_ROUNDS | DFAMIN_FLAG_INCREMENTAL_ROUNDS)) &&
                ((J.flags & DFAMIN_FLAG_MASKED_ROUNDS) ||
                 (count > kCacheMaxBlocks &&
                  (2ll * nlead_round <= (long long)n ||
                   moved_last * 4ull * (unsigned long long)max(ncols, 1) <= (unsigned long long)n)));
            const bool incr = !masked && have_rows && !leader_mode &&
                              !(J.flags & DFAMIN_FLAG_FULL_ROUNDS) &&
                              ((J.flags & DFAMIN_FLAG_INCREMENTAL_ROUNDS) ||
                               moved_last * 4ull * (unsigned long long)max(ncols, 1) <=
                                   (unsigned long long)n);
            // ---- phase A: empty the slots of last round's groups (listed in phase C by each
            //      group's smallest state), then leaders publish rows
            {
                const int nlead = nlead_cur;
                const int gid = rank * (int)blockDim.x + (int)threadIdx.x;
                for (int i = lead_reset_from + gid; i < nlead; i += T * (int)blockDim.x) {
                    if (leader_mode) J.naive_new[__ldcg(&J.lead_slot[i])] = 0x7fffffff;
                    else J.table[__ldcg(&J.lead_slot[i])] = kEmptySlot;
                }
                lead_reset_from = nlead;
                phase_leaders<KC>(J, rank, T, nlead, ncols, passes, incr, masked);
            }
            __syncthreads();
            if (threadIdx.x == 0) { s_claims = 0; s_cnt = 0; s_rst = 0; s_heads = 0; }
            if (!team_barrier(ts)) goto done;
            trace_mark(J, tw, passes, 4);

            // ---- phase B: signatures, comparison with the leader, regrouping of the rest
            bool use_cache = false;
            if constexpr (KC > 0) {
                extern __shared__ __align__(16) unsigned char dsm[];
                auto& cache = *reinterpret_cast<CtaCache<RowOf<KC>::SS>*>(dsm);
                use_cache = !leader_mode && !masked && count <= kCacheMaxBlocks;
                if (use_cache) {
                    cache_clear(cache);
                    __syncthreads();
                    phase_members_cached<KC>(J, c0, c1, &s_claims, &s_cnt, cache, &s_heads,
                                             passes, incr);
                } else {
                    phase_members<KC>(J, c0, c1, ncols, &s_claims, &s_cnt, &s_heads, passes,
                                      incr, masked);
                }
            } else {
                phase_members<KC>(J, c0, c1, ncols, &s_claims, &s_cnt, &s_heads, passes, incr,
                                  masked);
            }
            __syncthreads();
            {
                const int cl = leader_mode ? s_cnt : s_claims;   // leader mode: moved states
                if (threadIdx.x == 0 && cl) atomicAdd(&J.ctrl->claims, (unsigned long long)cl);
                if (threadIdx.x == 0 && s_cnt)
                    atomicAdd(&J.ctrl->moved, (unsigned long long)s_cnt);
                if (threadIdx.x == 0) J.cta_cnt[rank] = s_heads;
            }
            if (!team_barrier(ts, J.ctrl, &s_snap)) goto done;
            trace_mark(J, tw, passes, 5);

            const unsigned long long claims_now = s_snap.claims;
            const int new_groups = (int)(claims_now - claims_seen);
            claims_seen = claims_now;
            const unsigned long long moved_now = s_snap.moved;
            moved_last = moved_now - moved_seen;
            moved_seen = moved_now;
            if (new_groups == 0) {                    // partition unchanged: stable
                heads_valid = true;
                break;
            }

            // ---- phase C: moved states take their group's smallest state as id; that state
            //      becomes a leader and lists the group's slot to be emptied next round
            {
                const int cnt = s_cnt;
                if constexpr (KC > 0) {
                    constexpr int SS = RowOf<KC>::SS;
                    extern __shared__ __align__(16) unsigned char dsm[];
                    auto& cache = *reinterpret_cast<CtaCache<SS>*>(dsm);
                    if (use_cache) {
                        for (int ci = threadIdx.x; ci < CtaCache<RowOf<KC>::SS>::kSlots;
                             ci += blockDim.x)
                            if (cache.gslot[ci] != kEmpty)
                                cache.gmin[ci] = slot_min(__ldcg(&J.table[cache.gslot[ci]]));
                        __syncthreads();
                    }
                    // four entries per thread per step: their group-table reads are
                    // independent and in flight together
                    for (int b = 0; b < cnt; b += 4 * (int)blockDim.x) {
                        int sv[4];
                        uint32_t slv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int i = b + u * (int)blockDim.x + (int)threadIdx.x;
                            sv[u] = -1;
                            slv[u] = 0;
                            if (i < cnt) {
                                sv[u] = __ldcs(&J.lst_s[c0 + i]);
                                slv[u] = __ldcs(&J.lst_slot[c0 + i]);
                            }
                        }
                        int mv[4], hv[4];
                        uint32_t gsv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            mv[u] = 0;
                            hv[u] = 0;
                            gsv[u] = slv[u];
                            if (sv[u] < 0) continue;
                            if (use_cache && (slv[u] & kCached)) {
                                const int ci = (int)(slv[u] & ~kCached);
                                mv[u] = cache.gmin[ci];
                                hv[u] = cache.head[ci];
                                gsv[u] = cache.gslot[ci];
                            } else if (leader_mode) {
                                mv[u] = ld_volatile(&J.naive_new[slv[u]]);
                            } else {
                                const unsigned long long w = __ldcg(&J.table[slv[u]]);
                                mv[u] = slot_min(w);
                                hv[u] = slot_head(w);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            // a new block: the block its smallest member left lost members
                            if (sv[u] >= 0 && mv[u] == sv[u] && !leader_mode) J.spl[hv[u]] = passes;
                            if (sv[u] >= 0) J.block[sv[u]] = mv[u];
                            append_pair(J, c0, &s_rst, sv[u] >= 0 && mv[u] == sv[u], sv[u],
                                        gsv[u]);
                        }
                    }
                } else {
                    for (int b = 0; b < cnt; b += blockDim.x) {
                        const int i = b + threadIdx.x;
                        bool lead = false;
                        uint32_t gs = 0;
                        int s = 0;
                        if (i < cnt) {
                            s = J.lst_s[c0 + i];
                            gs = J.lst_slot[c0 + i];
                            const int m = leader_mode ? ld_volatile(&J.naive_new[gs])
                                                      : slot_min(__ldcg(&J.table[gs]));
                            lead = (m == s);
                            // a new block: the block s left lost members this round
                            if (lead && !leader_mode) J.spl[__ldcg(&J.block[s])] = passes;
                            J.block[s] = m;
                        }
                        append_pair(J, c0, &s_rst, lead, s, gs);
                    }
                }
                // publish this CTA's new leaders to the global list (one atomic per CTA)
                __syncthreads();
                const int nnew = s_rst;
                if (threadIdx.x == 0) s_base = nnew ? atomicAdd(&J.ctrl->nlead, nnew) : 0;
                __syncthreads();
                const int lbase = s_base;
                for (int i = threadIdx.x; i < nnew; i += blockDim.x) {
                    J.lead[lbase + i] = J.stg[c0 + i];
                    J.lead_slot[lbase + i] = J.lst_rst[c0 + i];
                }
            }
            if (!team_barrier(ts, J.ctrl, &s_snap)) goto done;
            trace_mark(J, tw, passes, 6);
            nlead_cur = s_snap.nlead;
            count = leader_mode ? nlead_cur : count + new_groups;
            have_rows = !leader_mode;
        }
        if (ld_volatile(&J.ctrl->status) != 0) goto done;

        // ---- canonical ids: rank of each leader among leaders, in state order.  Chunks start
        //      at multiples of 32 states, so block[] is read as int4 (4 states per thread).
        //      The per-CTA leader counts come from the last round's members phase when that
        //      round moved nothing; otherwise they are counted here.
        if (!heads_valid) {
            int heads = 0;
            for (int s = c0 + 4 * (int)threadIdx.x; s < c1; s += 4 * blockDim.x) {
                if (s + 3 < c1) {
                    const int4 b = __ldcg(reinterpret_cast<const int4*>(J.block + s));
                    heads += (b.x == s) + (b.y == s + 1) + (b.z == s + 2) + (b.w == s + 3);
                } else {
                    for (int j = s; j < min(s + 4, c1); ++j) heads += (ld_blk(&J.block[j]) == j);
                }
            }
            heads = cta_sum(heads);
            if (threadIdx.x == 0) J.cta_cnt[rank] = heads;
            if (!team_barrier(ts)) goto done;
        }
        trace_mark(J, tw, passes, 7);
        int offset = 0;
        for (int r = threadIdx.x; r < rank; r += blockDim.x) offset += __ldcg(&J.cta_cnt[r]);
        offset = cta_sum(offset);
        int total = 0;
        if (rank == T - 1) {
            for (int r = threadIdx.x; r < T; r += blockDim.x) total += __ldcg(&J.cta_cnt[r]);
            total = cta_sum(total);
        }
        // the next step's block ids are in flight while this step is scanned
        int4 nb = make_int4(0, 0, 0, 0);
        if (c0 + 4 * (int)threadIdx.x + 3 < c1)
            nb = __ldcg(reinterpret_cast<const int4*>(J.block + c0 + 4 * (int)threadIdx.x));
        for (int base = c0; base < c1; base += 4 * blockDim.x) {
            const int s = base + 4 * (int)threadIdx.x;
            int f[4] = {0, 0, 0, 0};
            const int4 b = nb;
            if (s + 4 * (int)blockDim.x + 3 < c1)
                nb = __ldcg(reinterpret_cast<const int4*>(J.block + s + 4 * (int)blockDim.x));
            if (s + 3 < c1) {
                f[0] = b.x == s; f[1] = b.y == s + 1; f[2] = b.z == s + 2; f[3] = b.w == s + 3;
            } else {
                for (int j = 0; j < 4; ++j) f[j] = (s + j < c1) && (ld_blk(&J.block[s + j]) == s + j);
            }
            int tile_total;
            int pre = offset + cta_scan_count(f[0] + f[1] + f[2] + f[3], &tile_total);
            for (int j = 0; j < 4; ++j)
                if (f[j]) J.out_block[s + j] = pre++;
            offset += tile_total;
        }
        if (!team_barrier(ts)) goto done;
        // out_block is the caller's array (in a batch: at the DFA's offset), so its int4 access
        // is used only when it is 16-byte aligned; block[] is in the workspace (aligned)
        const bool out_aligned = ((uintptr_t)J.out_block & 15u) == 0 &&
                                 ((uintptr_t)J.out_host & 15u) == 0;
        const int step = 4 * (int)blockDim.x;
        int4 pb = make_int4(0, 0, 0, 0), po = make_int4(0, 0, 0, 0);
        {
            const int s0 = c0 + 4 * (int)threadIdx.x;
            if (s0 + 3 < c1 && out_aligned) {
                pb = __ldcg(reinterpret_cast<const int4*>(J.block + s0));
                po = __ldcg(reinterpret_cast<const int4*>(J.out_block + s0));
            }
        }
        for (int s = c0 + 4 * (int)threadIdx.x; s < c1; s += step) {
            // the next step's ids and ranks are in flight while this step's gathers run
            const int4 b = pb, o = po;
            if (s + step + 3 < c1 && out_aligned) {
                pb = __ldcg(reinterpret_cast<const int4*>(J.block + s + step));
                po = __ldcg(reinterpret_cast<const int4*>(J.out_block + s + step));
            }
            if (s + 3 < c1 && out_aligned) {
                int4 r;
                r.x = b.x == s ? o.x : __ldcg(&J.out_block[b.x]);
                r.y = b.y == s + 1 ? o.y : __ldcg(&J.out_block[b.y]);
                r.z = b.z == s + 2 ? o.z : __ldcg(&J.out_block[b.z]);
                r.w = b.w == s + 3 ? o.w : __ldcg(&J.out_block[b.w]);
                // end-to-end calls: the labels go straight to host memory (the device array
                // keeps the leaders' ranks, the only entries gathered here)
                *reinterpret_cast<int4*>(J.out_host ? J.out_host + s : J.out_block + s) = r;
            } else {
                for (int j = s; j < min(s + 4, c1); ++j) {
                    const int L = ld_blk(&J.block[j]);
                    const int v = __ldcg(&J.out_block[L]);
                    if (J.out_host) J.out_host[j] = v;
                    else if (L != j) J.out_block[j] = v;
                }
            }
        }
        if (rank == T - 1 && threadIdx.x == 0) write_outputs(J, total, passes);
        if (J.trace) {                                // J.trace is uniform over the team
            if (!team_barrier(ts)) goto done;
            trace_mark(J, tw, passes, 8);
        }
        return;
    }
done:
    if (rank == 0 && threadIdx.x == 0) write_outputs(J, 0, passes);
}


// ------------------------------------------------------------------------------------------
// Small kernel: one CTA refines a DFA with n <= kSmallMaxStates entirely in shared memory.
// Shared table slots are 32-bit: [hash:16 | state:16], 0xffffffff = empty (n <= 65535).
// ------------------------------------------------------------------------------------------
static __device__ __forceinline__ int s_succ(const Job& J, int s, int c)
{
    return succ_col(J, s, c);
}

static __device__ bool s_tuples_equal(const Job& J, const int* sblock, int s, int t, int leader, int ncols)
{
    if (sblock[t] != leader) return false;
    for (int c = 0; c < ncols; ++c)
        if (sblock[s_succ(J, s, c)] != sblock[s_succ(J, t, c)]) return false;
    return true;
}

static __device__ void small_minimize(const Job& J, uint32_t cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = J.n, k = J.k;
    int* sblock = (int*)smem;                       // [n]
    int* spend = sblock + n;                        // [n] slot of a moved state, -1 otherwise
    uint32_t* stab = (uint32_t*)(spend + n);        // [cap]
    __shared__ int s_claims, s_bad;
    const bool closure = J.levels > 1;
    const bool elide = !(J.flags & DFAMIN_FLAG_KEEP_IDENTITY);
    const uint32_t smask = cap - 1;
    int passes = 0, count = 0;

    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    {
        bool bad = false;
        const int64_t total = (int64_t)n * k;
        for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
            const int v = __ldg(&J.delta[i]);
            if ((unsigned)v >= (unsigned)n) bad = true;
            if (closure && v != (int)(i / k)) J.nonid[i % k] = 1;
        }
        if (bad) s_bad = 1;
    }
    int mf = 0x7fffffff, mn = 0x7fffffff;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (is_accepting(J, s)) mf = min(mf, s); else mn = min(mn, s);
        spend[s] = -1;
    }
    mf = cta_min(mf);
    mn = cta_min(mn);
    if (s_bad) {
        if (threadIdx.x == 0) { set_status(J.ctrl, DFAMIN_EINVAL); write_outputs(J, 0, 0); }
        return;
    }
    for (int s = threadIdx.x; s < n; s += blockDim.x)
        sblock[s] = is_accepting(J, s) ? mf : mn;
    count = (mf != 0x7fffffff) + (mn != 0x7fffffff);
    int ncl_cols = 0;
    if (closure) {
        __syncthreads();   // nonid[] complete
        if (threadIdx.x == 0) {
            int m = 0;
            for (int a = 0; a < k; ++a)
                if (!elide || J.nonid[a]) J.cl_letter[m++] = a;
            J.ctrl->ncl_letters = m;
        }
        __syncthreads();
        ncl_cols = closure_build(J, 0, n, J.ctrl->ncl_letters, nullptr, false);
    }
    const int ncols = k + ncl_cols;
    __syncthreads();

    while (count < n) {
        if (passes >= J.max_passes) {
            if (threadIdx.x == 0) set_status(J.ctrl, DFAMIN_ENOCONVERGE);
            break;
        }
        ++passes;
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) stab[i] = 0xffffffffu;
        if (threadIdx.x == 0) s_claims = 0;
        __syncthreads();
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const int L = sblock[s];
            if (L == s) continue;
            uint64_t h = hash_begin(L);
            bool same = true;
            for (int c = 0; c < ncols; ++c) {
                const int b = sblock[s_succ(J, s, c)];
                if (same) same = (b == sblock[s_succ(J, L, c)]);
                h = hash_step(h, b);
            }
            if (same) continue;
            h = hash_final(h, L, J.flags);
            const uint32_t tag = (uint32_t)(h >> 48);
            const uint32_t mine = (tag << 16) | (uint32_t)s;
            uint32_t idx = (uint32_t)h & smask;
            uint32_t probe = 0;
            for (; probe <= smask; ++probe) {
                uint32_t w = stab[idx];
                if (w == 0xffffffffu) {
                    w = atomicCAS(&stab[idx], 0xffffffffu, mine);
                    if (w == 0xffffffffu) { atomicAdd(&s_claims, 1); break; }
                }
                if ((w >> 16) == tag) {
                    const int t = (int)(w & 0xffffu);
                    if (s_tuples_equal(J, sblock, s, t, L, ncols)) {
                        if (s < t) atomicMin(&stab[idx], mine);
                        break;
                    }
                }
                idx = (idx + 1) & smask;
            }
            if (probe > smask) { set_status(J.ctrl, DFAMIN_EPROBE); break; }
            spend[s] = (int)idx;
        }
        __syncthreads();
        const int new_groups = s_claims;
        if (ld_volatile(&J.ctrl->status) != 0 || new_groups == 0) break;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const int slot = spend[s];
            if (slot >= 0) { sblock[s] = (int)(stab[slot] & 0xffffu); spend[s] = -1; }
        }
        __syncthreads();
        count += new_groups;
    }
    __syncthreads();
    if (ld_volatile(&J.ctrl->status) != 0) {
        if (threadIdx.x == 0) write_outputs(J, 0, passes);
        return;
    }
    // canonical ids: ranks of leaders (kept in spend[]), then every state takes its leader's
    int offset = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const int head = (s < n) && (sblock[s] == s);
        int tile_total;
        const int pre = cta_scan_flag(head, &tile_total);
        if (head) spend[s] = offset + pre;
        offset += tile_total;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) J.out_block[s] = spend[sblock[s]];
    if (threadIdx.x == 0) write_outputs(J, offset, passes);
}

// ------------------------------------------------------------------------------------------
// Medium kernel: one CTA of kMediumThreads threads refines a DFA with n <= kMediumMaxStates
// (no closure), by signature rounds or by the leader election of Alg. 2.  Block ids and delta live in shared memory as 16-bit values (exact, as
// n <= 65535); the group table (64-bit slots, as in the team kernel) and the list of moved
// states are in global memory.  Phases are separated by __syncthreads only, so a round costs
// a few microseconds: for deep refinement (about one block split per round) this beats the
// multi-CTA kernel, whose rounds need three grid barriers.
// ------------------------------------------------------------------------------------------
constexpr int kMediumThreads = 1024;
constexpr int kMediumMaxStates = 65535;

static __device__ bool m_rows_equal(const uint16_t* sb, const uint16_t* sd, int k, int s, int t)
{
    for (int c = 0; c < k; ++c)
        if (sb[sd[s * k + c]] != sb[sd[t * k + c]]) return false;
    return true;
}

static __device__ void medium_minimize(const Job& J)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = J.n, k = J.k;
    uint16_t* sb = reinterpret_cast<uint16_t*>(smem);     // [n] leader ids
    uint16_t* sd = sb + n;                                 // [n*k] delta
    __shared__ int s_claims, s_cnt, s_bad;
    int passes = 0, count = 0;

    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    {
        bool bad = false;
        const int64_t total = (int64_t)n * k;
        for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
            const int v = __ldg(&J.delta[i]);
            if ((unsigned)v >= (unsigned)n) bad = true;
            sd[i] = (uint16_t)v;
        }
        if (bad) s_bad = 1;
    }
    const bool leader_mode = J.algo == DFAMIN_ALG_LEADER;
    if (leader_mode)
        for (int i = threadIdx.x; i < n; i += blockDim.x) J.naive_new[i] = 0x7fffffff;
    else
        for (uint64_t i = threadIdx.x; i <= (uint64_t)J.mask; i += blockDim.x)
            J.table[i] = kEmptySlot;
    int mf = 0x7fffffff, mn = 0x7fffffff;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (is_accepting(J, s)) mf = min(mf, s); else mn = min(mn, s);
    }
    mf = cta_min(mf);
    mn = cta_min(mn);
    if (s_bad) {
        if (threadIdx.x == 0) { set_status(J.ctrl, DFAMIN_EINVAL); write_outputs(J, 0, 0); }
        return;
    }
    for (int s = threadIdx.x; s < n; s += blockDim.x)
        sb[s] = (uint16_t)(is_accepting(J, s) ? mf : mn);
    count = (mf != 0x7fffffff) + (mn != 0x7fffffff);
    __syncthreads();

    // signature rounds stop once every block is a singleton; Alg. 2 runs until a round
    // changes nothing
    while (leader_mode || count < n) {
        if (passes >= J.max_passes) {
            if (threadIdx.x == 0) set_status(J.ctrl, DFAMIN_ENOCONVERGE);
            break;
        }
        ++passes;
        if (threadIdx.x == 0) { s_claims = 0; s_cnt = 0; }
        __syncthreads();
        // members: a state whose successors' ids differ from its leader's regroups by its full
        // signature in the global table (slot = (min << 32) | representative; equality is
        // decided on the rows, regathered from shared memory)
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const int L = sb[s];
            if (L == s) continue;
            bool same = true;
            for (int c = 0; c < k; ++c) same = same && sb[sd[s * k + c]] == sb[sd[L * k + c]];
            if (same) continue;
            if (leader_mode) {
                // Alg. 2: the states that differ from L form one new block, led by the
                // smallest of them
                if (atomicMin(&J.naive_new[L], s) == 0x7fffffff) atomicAdd(&s_claims, 1);
                const int pos = atomicAdd(&s_cnt, 1);
                J.lst_s[pos] = s;
                J.lst_slot[pos] = (uint32_t)L;
                continue;
            }
            uint64_t h = hash_begin(L);
            for (int c = 0; c < k; ++c) h = hash_step(h, sb[sd[s * k + c]]);
            h = hash_final(h, L, J.flags);
            uint32_t idx = (uint32_t)h & J.mask;
            uint32_t probe = 0;
            for (; probe <= J.mask; ++probe) {
                unsigned long long w = ld_acquire_u64(&J.table[idx]);
                if (w == kEmptySlot) {
                    w = atomicCAS(&J.table[idx], kEmptySlot, slot_word(s, s));
                    if (w == kEmptySlot) { atomicAdd(&s_claims, 1); break; }
                }
                const int rep = slot_rep(w);
                if (sb[rep] == L && m_rows_equal(sb, sd, k, s, rep)) {
                    if (s < slot_min(w)) atomicMin(&J.table[idx], slot_word(s, rep));
                    break;
                }
                idx = (idx + 1) & J.mask;
            }
            if (probe > J.mask) { set_status(J.ctrl, DFAMIN_EPROBE); break; }
            const int pos = atomicAdd(&s_cnt, 1);
            J.lst_s[pos] = s;
            J.lst_slot[pos] = idx;
        }
        __syncthreads();
        const int claims = s_claims, cnt = s_cnt;
        if (ld_volatile(&J.ctrl->status) != 0 || claims == 0) break;
        // moves: every listed state takes its group's smallest state as id
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t slot = __ldcg(&J.lst_slot[i]);
            sb[__ldcg(&J.lst_s[i])] =
                (uint16_t)(leader_mode ? __ldcg(&J.naive_new[slot])
                                       : slot_min(__ldcg(&J.table[slot])));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t slot = __ldcg(&J.lst_slot[i]);
            if (leader_mode) J.naive_new[slot] = 0x7fffffff;
            else J.table[slot] = kEmptySlot;
        }
        __syncthreads();
        count += claims;
    }
    __syncthreads();
    if (ld_volatile(&J.ctrl->status) != 0) {
        if (threadIdx.x == 0) write_outputs(J, 0, passes);
        return;
    }
    // canonical ids: ranks of the leaders in state order, then every state takes its leader's
    int offset = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const int head = (s < n) && (sb[s] == s);
        int tile_total;
        const int pre = cta_scan_flag(head, &tile_total);
        if (head) J.stg[s] = offset + pre;
        offset += tile_total;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) J.out_block[s] = __ldcg(&J.stg[sb[s]]);
    if (threadIdx.x == 0) write_outputs(J, offset, passes);
}

}  // namespace dfamin_dev

// dfamin: signature-based partition refinement of DFA states on GB300 (sm_103a).
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

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "dfamin.h"

#define DFAMIN_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kThreads = 256;             // threads per CTA (team and small kernels)
constexpr int kMaxCtas = 8192;            // capacity of the per-CTA count array
constexpr uint32_t kEpochBits = 20;       // table epoch field width
constexpr uint32_t kEpochPeriod = (1u << kEpochBits) - 1;  // epochs 1..period, 0 = empty
constexpr int64_t kBarrierTimeoutNs = 4000000000ll;        // 4 s per CTA barrier
constexpr int kSmallMaxStates = 8192;     // largest n for the shared-memory kernel

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
    int pad[8];
};

struct Job {
    int32_t n, k;
    const int32_t* __restrict__ delta;   // [n*k] state-major, never written
    const uint32_t* __restrict__ accept; // bitmap
    int32_t* out_block;                  // [n]
    int32_t* nblocks_out;                // scalar
    int32_t* passes_out;                 // scalar or null
    int32_t* status_out;                 // scalar or null
    int32_t* block;                      // [n] leader ids
    int32_t* cl;                         // closure columns [ncl_letters*(levels-1)][n]
    int32_t* cl_letter;                  // [k] letters with closure columns (compacted)
    int32_t* nonid;                      // [k] 1 if letter is not the identity
    uint64_t* table;                     // [mask+1]
    int32_t* lst_s;                      // [n] changed states, per-CTA segments
    uint32_t* lst_slot;                  // [n] their table slots
    int32_t* cta_cnt;                    // [kMaxCtas]
    Ctrl* ctrl;
    uint32_t mask;                       // table capacity - 1
    int32_t levels;                      // closure levels (1 = no closure)
    int32_t max_passes;
    uint32_t flags;
    int64_t timeout_ns;
};

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ void set_status(Ctrl* c, int code) { atomicCAS(&c->status, 0, code); }

// splitmix64 finalizer (Steele, Lea & Flood 2014); the hash only steers the table probe.
__device__ __forceinline__ uint64_t fmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hash_begin(int leader)
{
    return fmix64((uint64_t)(uint32_t)leader * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull);
}
__device__ __forceinline__ uint64_t hash_step(uint64_t h, int b)
{
    return fmix64(h + 0x9E3779B97F4A7C15ull + (uint64_t)(uint32_t)b);
}
__device__ __forceinline__ uint64_t hash_final(uint64_t h, int leader, uint32_t flags)
{
    if (flags & DFAMIN_FLAG_HASH_CONSTANT) return 0;
    if (flags & DFAMIN_FLAG_HASH_BLOCK_ONLY) return hash_begin(leader);
    return h;
}

__device__ __forceinline__ int is_accepting(const uint32_t* acc, int s)
{
    return (int)((__ldg(&acc[s >> 5]) >> (s & 31)) & 1u);
}

// Successor of s under signature column c: the k letters, then the closure columns.
__device__ __forceinline__ int succ_col(const Job& J, int s, int c)
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

__device__ bool team_barrier(TeamSync& ts)
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
            unsigned sleep_ns = 32;
            for (;;) {
                if (ld_acquire_u64(ts.bar) >= target) break;
                if (ld_volatile(ts.status) != 0) { ok = 0; break; }
                if ((int64_t)(gtimer() - t0) > ts.timeout_ns) {
                    atomicCAS(ts.status, 0, (int)DFAMIN_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(sleep_ns);
                if (sleep_ns < 256) sleep_ns <<= 1;
            }
        }
        __threadfence();
        if (ld_volatile(ts.status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive prefix of a 0/1 flag over the CTA's threads; *total receives the CTA sum.
// Must be called by all threads of the CTA.
__device__ int cta_scan_flag(int flag, int* total)
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

__device__ int cta_sum(int v)
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

__device__ int cta_min(int v)
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
// Global hash table (team kernel).  Slot word: [epoch:20 | hash:12 | state:32]; a slot whose
// epoch differs from the round's epoch is empty.  All members of one group end in the same slot
// (a slot, once claimed in a round, never changes owner group) and its low word converges to
// the group's smallest state by atomicMin (the high word is equal for the whole group).
// ------------------------------------------------------------------------------------------
__device__ bool tuples_equal(const Job& J, int s, int t, int leader, int ncols)
{
    if (__ldcg(&J.block[t]) != leader) return false;
    for (int c = 0; c < ncols; ++c) {
        const int bs = __ldcg(&J.block[succ_col(J, s, c)]);
        const int bt = __ldcg(&J.block[succ_col(J, t, c)]);
        if (bs != bt) return false;
    }
    return true;
}

// Returns the slot of s's group, or UINT32_MAX after setting DFAMIN_EPROBE.
__device__ uint32_t table_insert(const Job& J, int s, int leader, uint64_t h, uint32_t epoch,
                                 int ncols, int* s_claims)
{
    const uint32_t tag = (epoch << 12) | (uint32_t)(h >> 52);
    const uint64_t mine = ((uint64_t)tag << 32) | (uint32_t)s;
    uint32_t idx = (uint32_t)h & J.mask;
    for (uint32_t probe = 0; probe <= J.mask; ++probe) {
        uint64_t w = ld_relaxed_u64(&J.table[idx]);
        while ((uint32_t)(w >> (64 - kEpochBits)) != epoch) {
            const uint64_t old = atomicCAS((unsigned long long*)&J.table[idx],
                                           (unsigned long long)w, (unsigned long long)mine);
            if (old == w) {
                atomicAdd(s_claims, 1);
                return idx;
            }
            w = old;
        }
        if ((uint32_t)(w >> 32) == tag) {
            const int t = (int)(uint32_t)w;
            if (t == s || tuples_equal(J, s, t, leader, ncols)) {
                if ((uint32_t)s < (uint32_t)t)
                    atomicMin((unsigned long long*)&J.table[idx], (unsigned long long)mine);
                return idx;
            }
        }
        idx = (idx + 1) & J.mask;
    }
    set_status(J.ctrl, DFAMIN_EPROBE);
    return 0xffffffffu;
}

// ------------------------------------------------------------------------------------------
// Team kernel body: one DFA refined by T co-resident CTAs; CTA `rank` owns states [c0, c1).
// ------------------------------------------------------------------------------------------
__device__ void write_outputs(const Job& J, int nblocks, int passes)
{
    const int st = ld_volatile(&J.ctrl->status);
    *J.nblocks_out = st ? -st : nblocks;
    if (J.passes_out) *J.passes_out = passes;
    if (J.status_out) *J.status_out = st;
}

__device__ void team_minimize(const Job& J, int rank, int T, TeamSync& ts)
{
    __shared__ int s_claims;
    __shared__ int s_cnt;
    const int n = J.n, k = J.k;
    const int chunk = (n + T - 1) / T;
    const int c0 = min(n, rank * chunk), c1 = min(n, c0 + chunk);
    const bool closure = J.levels > 1;
    const bool elide = !(J.flags & DFAMIN_FLAG_KEEP_IDENTITY);
    int passes = 0;

    // ---- phase V: validate delta rows, find the two initial leaders, mark identity letters
    {
        bool bad = false;
        const int64_t r0 = (int64_t)c0 * k, r1 = (int64_t)c1 * k;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const int v = __ldg(&J.delta[i]);
            if ((unsigned)v >= (unsigned)n) bad = true;
            if (closure && v != (int)(i / k)) J.nonid[i % k] = 1;
        }
        if (bad) set_status(J.ctrl, DFAMIN_EINVAL);
        int mf = 0x7fffffff, mn = 0x7fffffff;
        for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
            if (is_accepting(J.accept, s)) mf = min(mf, s); else mn = min(mn, s);
        }
        mf = cta_min(mf);
        mn = cta_min(mn);
        if (threadIdx.x == 0) {
            if (mf != 0x7fffffff) atomicMax(&J.ctrl->min_f_rev, n - mf);
            if (mn != 0x7fffffff) atomicMax(&J.ctrl->min_n_rev, n - mn);
        }
        // clear the hash table slice owned by this CTA
        const uint64_t cap = (uint64_t)J.mask + 1;
        const uint64_t per = (cap + T - 1) / T;
        const uint64_t t0 = min(cap, per * rank), t1 = min(cap, t0 + per);
        for (uint64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) J.table[i] = 0;
    }
    if (!team_barrier(ts)) goto done;

    // ---- phase I: initial partition P0 = {F, Q\F} as leader ids
    {
        const int rf = ld_volatile(&J.ctrl->min_f_rev), rn = ld_volatile(&J.ctrl->min_n_rev);
        const int lf = n - rf, ln = n - rn;
        for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x)
            J.block[s] = is_accepting(J.accept, s) ? lf : ln;
        if (closure && rank == 0 && threadIdx.x == 0) {
            int m = 0;
            for (int a = 0; a < k; ++a)
                if (!elide || ld_volatile(&J.nonid[a])) J.cl_letter[m++] = a;
            J.ctrl->ncl_letters = m;
        }
    }
    if (!team_barrier(ts)) goto done;

    {
        int count = (ld_volatile(&J.ctrl->min_f_rev) > 0) + (ld_volatile(&J.ctrl->min_n_rev) > 0);
        const int ncl = closure ? ld_volatile(&J.ctrl->ncl_letters) : 0;
        const int lv = J.levels - 1;

        // ---- closure levels (Alg. transPR): level i of letter a is level i-1 applied twice
        for (int i = 1; i <= lv && closure; ++i) {
            for (int j = 0; j < ncl; ++j) {
                const int a = __ldcg(&J.cl_letter[j]);
                int32_t* cur = J.cl + ((int64_t)j * lv + (i - 1)) * n;
                for (int q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
                    int t;
                    if (i == 1) {
                        t = __ldg(&J.delta[(int64_t)q * k + a]);
                        t = __ldg(&J.delta[(int64_t)t * k + a]);
                    } else {
                        const int32_t* prev = cur - n;   // level i-1 of the same letter
                        t = __ldcg(&prev[q]);
                        t = __ldcg(&prev[t]);
                    }
                    cur[q] = t;
                }
            }
            if (!team_barrier(ts)) goto done;
        }

        const int ncols = k + ncl * lv;
        const int max_passes = J.max_passes;
        unsigned long long claims_seen = 0;
        while (count < n) {
            if (passes >= max_passes) {
                set_status(J.ctrl, DFAMIN_ENOCONVERGE);
                break;
            }
            ++passes;
            const uint32_t epoch = (uint32_t)((passes - 1) % kEpochPeriod) + 1;
            if (passes > 1 && epoch == 1) {   // epoch wrapped: clear the table slice again
                const uint64_t cap = (uint64_t)J.mask + 1;
                const uint64_t per = (cap + T - 1) / T;
                const uint64_t t0 = min(cap, per * rank), t1 = min(cap, t0 + per);
                for (uint64_t x = t0 + threadIdx.x; x < t1; x += blockDim.x) J.table[x] = 0;
                if (!team_barrier(ts)) goto done;
            }
            if (threadIdx.x == 0) { s_claims = 0; s_cnt = 0; }
            __syncthreads();

            // ---- phase B: signatures, comparison with the leader, regrouping of the rest
            for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
                const int L = __ldcg(&J.block[s]);
                if (L == s) continue;                 // a leader keeps its id
                uint64_t h = hash_begin(L);
                bool same = true;
                for (int c = 0; c < ncols; ++c) {
                    const int b = __ldcg(&J.block[succ_col(J, s, c)]);
                    if (same) same = (b == __ldcg(&J.block[succ_col(J, L, c)]));
                    h = hash_step(h, b);
                }
                if (same) continue;                   // T(s) == T(leader): id unchanged
                h = hash_final(h, L, J.flags);
                const uint32_t slot = table_insert(J, s, L, h, epoch, ncols, &s_claims);
                if (slot == 0xffffffffu) break;
                const int pos = atomicAdd(&s_cnt, 1);
                J.lst_s[c0 + pos] = s;
                J.lst_slot[c0 + pos] = slot;
            }
            __syncthreads();
            if (threadIdx.x == 0 && s_claims) atomicAdd(&J.ctrl->claims, (unsigned long long)s_claims);
            if (!team_barrier(ts)) goto done;

            const unsigned long long claims_now = ld_acquire_u64(&J.ctrl->claims);
            const int new_groups = (int)(claims_now - claims_seen);
            claims_seen = claims_now;
            if (new_groups == 0) break;               // partition unchanged: stable

            // ---- phase C: moved states take their group's smallest state as id
            const int cnt = s_cnt;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int s = J.lst_s[c0 + i];
                const uint32_t slot = J.lst_slot[c0 + i];
                J.block[s] = (int)(uint32_t)ld_relaxed_u64(&J.table[slot]);
            }
            if (!team_barrier(ts)) goto done;
            count += new_groups;
        }
        if (ld_volatile(&J.ctrl->status) != 0) goto done;

        // ---- canonical ids: rank of each leader among leaders, in state order
        int heads = 0;
        for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x)
            heads += (__ldcg(&J.block[s]) == s);
        heads = cta_sum(heads);
        if (threadIdx.x == 0) J.cta_cnt[rank] = heads;
        if (!team_barrier(ts)) goto done;
        int offset = 0;
        for (int r = threadIdx.x; r < rank; r += blockDim.x) offset += __ldcg(&J.cta_cnt[r]);
        offset = cta_sum(offset);
        int total = 0;
        if (rank == T - 1) {
            for (int r = threadIdx.x; r < T; r += blockDim.x) total += __ldcg(&J.cta_cnt[r]);
            total = cta_sum(total);
        }
        for (int base = c0; base < c1; base += blockDim.x) {
            const int s = base + threadIdx.x;
            const int head = (s < c1) && (__ldcg(&J.block[s]) == s);
            int tile_total;
            const int pre = cta_scan_flag(head, &tile_total);
            if (head) J.out_block[s] = offset + pre;
            offset += tile_total;
        }
        if (!team_barrier(ts)) goto done;
        for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
            const int L = __ldcg(&J.block[s]);
            if (L != s) J.out_block[s] = __ldcg(&J.out_block[L]);
        }
        if (rank == T - 1 && threadIdx.x == 0) write_outputs(J, total, passes);
        return;
    }
done:
    if (rank == 0 && threadIdx.x == 0) write_outputs(J, 0, passes);
}

__global__ void __launch_bounds__(kThreads) team_kernel(Job J)
{
    TeamSync ts{&J.ctrl->bar, &J.ctrl->status, (unsigned long long)gridDim.x, 0ull, J.timeout_ns};
    team_minimize(J, blockIdx.x, gridDim.x, ts);
}

// ------------------------------------------------------------------------------------------
// Small kernel: one CTA refines a DFA with n <= kSmallMaxStates entirely in shared memory.
// Shared table slots are 32-bit: [hash:16 | state:16], 0xffffffff = empty (n <= 65535).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int s_succ(const Job& J, int s, int c)
{
    return succ_col(J, s, c);
}

__device__ bool s_tuples_equal(const Job& J, const int* sblock, int s, int t, int leader, int ncols)
{
    if (sblock[t] != leader) return false;
    for (int c = 0; c < ncols; ++c)
        if (sblock[s_succ(J, s, c)] != sblock[s_succ(J, t, c)]) return false;
    return true;
}

__device__ void small_minimize(const Job& J, uint32_t cap)
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
        if (is_accepting(J.accept, s)) mf = min(mf, s); else mn = min(mn, s);
        spend[s] = -1;
    }
    mf = cta_min(mf);
    mn = cta_min(mn);
    if (s_bad) {
        if (threadIdx.x == 0) { set_status(J.ctrl, DFAMIN_EINVAL); write_outputs(J, 0, 0); }
        return;
    }
    for (int s = threadIdx.x; s < n; s += blockDim.x)
        sblock[s] = is_accepting(J.accept, s) ? mf : mn;
    count = (mf != 0x7fffffff) + (mn != 0x7fffffff);
    int ncl = 0;
    const int lv = J.levels - 1;
    if (closure) {
        __syncthreads();   // nonid[] complete
        if (threadIdx.x == 0) {
            int m = 0;
            for (int a = 0; a < k; ++a)
                if (!elide || J.nonid[a]) J.cl_letter[m++] = a;
            J.ctrl->ncl_letters = m;
        }
        __syncthreads();
        ncl = J.ctrl->ncl_letters;
        for (int i = 1; i <= lv; ++i) {
            for (int j = 0; j < ncl; ++j) {
                const int a = J.cl_letter[j];
                int32_t* cur = J.cl + ((int64_t)j * lv + (i - 1)) * n;
                for (int q = threadIdx.x; q < n; q += blockDim.x) {
                    int t;
                    if (i == 1) {
                        t = __ldg(&J.delta[(int64_t)q * k + a]);
                        t = __ldg(&J.delta[(int64_t)t * k + a]);
                    } else {
                        const int32_t* prev = cur - n;   // level i-1 of the same letter
                        t = prev[q];
                        t = prev[t];
                    }
                    cur[q] = t;
                }
            }
            __syncthreads();
        }
    }
    const int ncols = k + ncl * lv;
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

__global__ void __launch_bounds__(kThreads) small_kernel(Job J, uint32_t cap)
{
    small_minimize(J, cap);
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline uint32_t next_pow2_u32(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return (uint32_t)p;
}

inline int floor_log2(int64_t n)
{
    int l = 0;
    while (((int64_t)1 << (l + 1)) <= n) ++l;
    return l;
}

struct Layout {
    size_t ctrl, cta_cnt, nonid, zero_end;  // [ctrl .. zero_end) is zeroed per launch
    size_t block, lst_s, lst_slot, table, cl, cl_letter, total;
    uint32_t cap;
    int levels;
};

Layout make_layout(int32_t n, int32_t k, const dfamin_options& o)
{
    Layout L{};
    const size_t A = 256;
    size_t off = 0;
    L.ctrl = off; off = align_up(off + sizeof(Ctrl), A);
    L.cta_cnt = off; off = align_up(off + sizeof(int32_t) * kMaxCtas, A);
    L.nonid = off; off = align_up(off + sizeof(int32_t) * (size_t)(k > 0 ? k : 1), A);
    L.zero_end = off;
    L.cl_letter = off; off = align_up(off + sizeof(int32_t) * (size_t)(k > 0 ? k : 1), A);
    L.block = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.lst_s = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.lst_slot = off; off = align_up(off + sizeof(uint32_t) * (size_t)n, A);
    L.cap = next_pow2_u32((uint64_t)n + (uint64_t)n / 2 + 64);
    L.table = off; off = align_up(off + sizeof(uint64_t) * (size_t)L.cap, A);
    L.levels = (o.closure == DFAMIN_CLOSURE_ON) ? floor_log2(n) + 1 : 1;
    L.cl = off;
    off = align_up(off + sizeof(int32_t) * (size_t)n * (size_t)k * (size_t)(L.levels - 1), A);
    L.total = off;
    return L;
}

dfamin_status check_options(const dfamin_options& o)
{
    if (o.closure != DFAMIN_CLOSURE_OFF && o.closure != DFAMIN_CLOSURE_ON) return DFAMIN_EINVAL;
    if (o.max_passes < 0 || o.ctas < 0 || o.smem_states < 0) return DFAMIN_EINVAL;
    if (o.reserved[0] || o.reserved[1] || o.reserved[2]) return DFAMIN_EINVAL;
    return DFAMIN_OK;
}

struct DeviceInfo {
    int sms = 0;
    int team_blocks_per_sm = 0;
    size_t smem_optin = 0;
};

std::mutex g_mu;
std::map<int, DeviceInfo> g_dev;

// Last CUDA failure seen by this thread (dfamin_last_cuda_error).
thread_local char g_last_error[256] = "";

bool cuda_ok(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return true;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", what, cudaGetErrorString(e),
             (int)e);
    return false;
}

dfamin_status device_info(DeviceInfo* out)
{
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return DFAMIN_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) { *out = it->second; return DFAMIN_OK; }
    DeviceInfo d;
    int v = 0;
    if (!cuda_ok(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev),
                 "cudaDeviceGetAttribute(SMs)"))
        return DFAMIN_ECUDA;
    if (!cuda_ok(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                 "cudaDeviceGetAttribute(smem)"))
        return DFAMIN_ECUDA;
    cudaFuncAttributes fa;
    if (!cuda_ok(cudaFuncGetAttributes(&fa, small_kernel), "cudaFuncGetAttributes"))
        return DFAMIN_ECUDA;
    d.smem_optin = (size_t)v > fa.sharedSizeBytes ? (size_t)v - fa.sharedSizeBytes : 0;
    if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.team_blocks_per_sm,
                                                               team_kernel, kThreads, 0),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
        return DFAMIN_ECUDA;
    if (!cuda_ok(cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)d.smem_optin),
                 "cudaFuncSetAttribute(small_kernel)"))
        return DFAMIN_ECUDA;
    g_dev[dev] = d;
    *out = d;
    return DFAMIN_OK;
}

size_t small_smem_bytes(int32_t n, uint32_t* cap_out)
{
    const uint32_t cap = next_pow2_u32((uint64_t)n + (uint64_t)n / 2 + 32);
    if (cap_out) *cap_out = cap;
    return sizeof(int32_t) * 2 * (size_t)n + sizeof(uint32_t) * (size_t)cap;
}

dfamin_status launch_one(int32_t n, int32_t k, const int32_t* delta, const uint32_t* accept,
                         int32_t* out_block, int32_t* nblocks, const dfamin_options& o,
                         void* ws, size_t ws_bytes, int32_t* passes, int32_t* status,
                         cudaStream_t stream)
{
    if (n < 1 || k < 0 || (int64_t)n * (int64_t)k >= ((int64_t)1 << 40)) return DFAMIN_EINVAL;
    if ((k > 0 && !delta) || !accept || !out_block || !nblocks || !ws) return DFAMIN_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return DFAMIN_EINVAL;
    dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    const Layout L = make_layout(n, k, o);
    if (ws_bytes < L.total) return DFAMIN_ENOMEM;
    DeviceInfo di;
    st = device_info(&di);
    if (st != DFAMIN_OK) return st;

    unsigned char* base = (unsigned char*)ws;
    Job J{};
    J.n = n;
    J.k = k;
    J.delta = delta;
    J.accept = accept;
    J.out_block = out_block;
    J.nblocks_out = nblocks;
    J.passes_out = passes;
    J.status_out = status;
    J.ctrl = (Ctrl*)(base + L.ctrl);
    J.cta_cnt = (int32_t*)(base + L.cta_cnt);
    J.nonid = (int32_t*)(base + L.nonid);
    J.cl_letter = (int32_t*)(base + L.cl_letter);
    J.block = (int32_t*)(base + L.block);
    J.lst_s = (int32_t*)(base + L.lst_s);
    J.lst_slot = (uint32_t*)(base + L.lst_slot);
    J.table = (uint64_t*)(base + L.table);
    J.mask = L.cap - 1;
    J.cl = (int32_t*)(base + L.cl);
    J.levels = L.levels;
    J.max_passes = o.max_passes > 0 ? o.max_passes : (n < 0x7fffffff ? n + 1 : n);
    J.flags = o.flags;
    J.timeout_ns = kBarrierTimeoutNs;

    if (!cuda_ok(cudaMemsetAsync(base + L.ctrl, 0, L.zero_end - L.ctrl, stream),
                 "cudaMemsetAsync(ctrl)"))
        return DFAMIN_ECUDA;

    const int small_limit = o.smem_states > 0 ? o.smem_states : 4096;
    uint32_t scap = 0;
    const size_t smem = small_smem_bytes(n, &scap);
    if (n <= small_limit && n <= kSmallMaxStates && smem <= di.smem_optin) {
        small_kernel<<<1, kThreads, smem, stream>>>(J, scap);
        return cuda_ok(cudaGetLastError(), "small_kernel launch") ? DFAMIN_OK : DFAMIN_ECUDA;
    }
    int max_ctas = di.sms * di.team_blocks_per_sm;
    if (max_ctas > kMaxCtas) max_ctas = kMaxCtas;
    int ctas = o.ctas > 0 ? o.ctas : max_ctas;
    // at least ~2 states per thread per CTA: small DFAs use fewer CTAs (cheaper barriers)
    const int64_t want = ((int64_t)n + 2 * kThreads - 1) / (2 * kThreads);
    if (o.ctas == 0 && want < ctas) ctas = (int)(want > 0 ? want : 1);
    if (ctas > max_ctas) ctas = max_ctas;
    void* args[] = {&J};
    if (!cuda_ok(cudaLaunchCooperativeKernel((const void*)team_kernel, dim3(ctas),
                                             dim3(kThreads), args, 0, stream),
                 "team_kernel cooperative launch"))
        return DFAMIN_ECUDA;
    return DFAMIN_OK;
}

// Library-owned workspaces for dfamin_minimize: one per (device, stream).
struct OwnedWs {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, OwnedWs> g_ws;

}  // namespace

DFAMIN_API void dfamin_default_options(dfamin_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->closure = DFAMIN_CLOSURE_OFF;
}

DFAMIN_API dfamin_status dfamin_workspace_size(int32_t n, int32_t k, const dfamin_options* opt,
                                               size_t* bytes)
{
    if (n < 1 || k < 0 || !bytes) return DFAMIN_EINVAL;
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    const dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    *bytes = make_layout(n, k, o).total;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_minimize_ex(int32_t n, int32_t k, const int32_t* delta,
                                            const uint32_t* accept, int32_t* out_block,
                                            int32_t* nblocks, const dfamin_options* opt,
                                            void* workspace, size_t workspace_bytes,
                                            int32_t* passes, int32_t* status,
                                            dfamin_stream_t stream)
{
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    return launch_one(n, k, delta, accept, out_block, nblocks, o, workspace, workspace_bytes,
                      passes, status, (cudaStream_t)stream);
}

DFAMIN_API dfamin_status dfamin_minimize(int32_t n, int32_t k, const int32_t* delta,
                                         const uint32_t* accept, int32_t* out_block,
                                         int32_t* nblocks, dfamin_stream_t stream)
{
    if (n < 1 || k < 0) return DFAMIN_EINVAL;
    dfamin_options o;
    dfamin_default_options(&o);
    const size_t need = make_layout(n, k, o).total;
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return DFAMIN_ECUDA;
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        OwnedWs& w = g_ws[std::make_pair(dev, (cudaStream_t)stream)];
        if (w.bytes < need) {
            if (w.ptr) {
                if (!cuda_ok(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize"))
                    return DFAMIN_ECUDA;
                cudaFree(w.ptr);
                w.ptr = nullptr;
                w.bytes = 0;
            }
            if (!cuda_ok(cudaMalloc(&w.ptr, need), "cudaMalloc(workspace)")) return DFAMIN_ENOMEM;
            w.bytes = need;
        }
        ws = w.ptr;
    }
    return launch_one(n, k, delta, accept, out_block, nblocks, o, ws, need, nullptr, nullptr,
                      (cudaStream_t)stream);
}

DFAMIN_API const char* dfamin_last_cuda_error(void) { return g_last_error; }

DFAMIN_API const char* dfamin_status_string(dfamin_status s)
{
    switch (s) {
    case DFAMIN_OK: return "DFAMIN_OK";
    case DFAMIN_EINVAL: return "DFAMIN_EINVAL";
    case DFAMIN_ENOMEM: return "DFAMIN_ENOMEM";
    case DFAMIN_ECUDA: return "DFAMIN_ECUDA";
    case DFAMIN_ETIMEOUT: return "DFAMIN_ETIMEOUT";
    case DFAMIN_ENOCONVERGE: return "DFAMIN_ENOCONVERGE";
    case DFAMIN_EPROBE: return "DFAMIN_EPROBE";
    }
    return "DFAMIN_UNKNOWN";
}

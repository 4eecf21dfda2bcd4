// Reachability from the initial state and the quotient automaton (arXiv 2410.22764, Sec. 2:
// minimization merges indistinguishable states and deletes the states that no word leads to
// from q0; the paper treats the deletion as a pre-processing step and its algorithms assume a
// fully reachable DFA).
//
//   reach_kernel     breadth-first search from q0 over a visited bitmap, then an
//                    order-preserving renumbering of the reached states and, optionally, the
//                    sub-DFA they induce.  One cooperative launch; levels meet at bounded
//                    barriers.  A thread that claims a new state keeps exploring from it with a
//                    small private stack before handing the rest to the next level: up to
//                    kReachBudgetChain states per frontier entry while the frontier stays tiny
//                    (a chain of length L then takes about L / 256 levels instead of L), up to
//                    kReachBudgetWide once it grows (so a branching graph spreads over all
//                    threads instead of being walked by a few).
//   quotient_kernel  the minimal DFA from a partition: every class (restricted to reachable
//                    states when a renumbering is given) is represented by its smallest member;
//                    classes are numbered in the order of their representatives, and
//                    delta'(B, a) = class of delta(rep(B), a).
//
// dfamin_minimal_dfa chains reach_kernel, the refinement kernels on the whole DFA and
// quotient_kernel on one stream with no host round trip.  Refining the whole DFA instead of
// the reachable sub-DFA gives the same classes on the reachable states (language equivalence of
// two states depends only on the states reachable from them) and keeps every size known on the
// host.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "dfamin.h"
#include "refine.cuh"
#include "host_common.h"

namespace dfamin_dev {

namespace cg = cooperative_groups;

constexpr int kReachStack = 16;      // private DFS stack of a thread (entries)
constexpr int kReachBudgetChain = 256;   // states a frontier entry may expand on a chain
constexpr int kReachBudgetWide = 8;      // ... and on a graph whose frontier grows

struct ReachCtrl {
    unsigned long long bar;          // team barrier counter
    int status;
    int fcnt[3];                     // frontier sizes, rotating by level % 3
};

struct ReachJob {
    int32_t n, k, q0;
    const int32_t* delta;
    const uint32_t* accept;
    uint32_t* vis;                   // [(n+31)/32] visited bitmap, zeroed before the launch
    int32_t* f0;                     // [n] frontier of even levels
    int32_t* f1;                     // [n] frontier of odd levels
    int32_t* cta_sum;                // [grid]
    int32_t* newid;                  // [n] out: rank among reached states, or -1
    int32_t* out_delta;              // [count*k] out or null: induced sub-DFA
    uint32_t* out_accept;            // [(n+31)/32] out (zeroed before the launch) or null
    int32_t* count_out;              // device scalar or null
    int32_t* status_out;             // device scalar or null
    ReachCtrl* ctrl;
    int64_t timeout_ns;
};

static __device__ __forceinline__ void reach_fail(ReachCtrl* c, int code)
{
    atomicCAS(&c->status, 0, code);
}

// Appends v to a frontier: one atomic per group of lanes that append together.
static __device__ __forceinline__ void frontier_push(int32_t* G, int* cnt, int v)
{
    cg::coalesced_group g = cg::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(cnt, (int)g.size());
    base = g.shfl(base, 0);
    G[base + (int)g.thread_rank()] = v;
}

// Expands frontier entry s0: every successor not yet visited is claimed (atomicOr on the
// bitmap); claimed states are explored by this thread while its budget lasts, the rest go to
// the next level.  Every state enters some frontier at most once, so a frontier holds <= n.
static __device__ void reach_expand(const ReachJob& R, int s0, int32_t* G, int* gcnt, int budget)
{
    int stack[kReachStack];
    int sp = 0;
    stack[sp++] = s0;
    while (sp > 0) {
        const int s = stack[--sp];
        if (budget == 0) {
            frontier_push(G, gcnt, s);
            continue;
        }
        --budget;
        const int32_t* row = R.delta + (int64_t)s * R.k;
        for (int a = 0; a < R.k; ++a) {
            const int t = __ldg(&row[a]);
            if ((unsigned)t >= (unsigned)R.n) {
                reach_fail(R.ctrl, DFAMIN_EINVAL);
                continue;
            }
            const uint32_t bit = 1u << (t & 31);
            if (ld_relaxed_u32(&R.vis[t >> 5]) & bit) continue;
            if (atomicOr(&R.vis[t >> 5], bit) & bit) continue;
            if (sp < kReachStack) stack[sp++] = t;
            else frontier_push(G, gcnt, t);
        }
    }
}

__global__ void __launch_bounds__(kTeamThreads) reach_kernel(ReachJob R)
{
    TeamSync ts{&R.ctrl->bar, &R.ctrl->status, (unsigned long long)gridDim.x, 0ull,
                R.timeout_ns};
    const int rank = blockIdx.x, T = gridDim.x;
    const int gid = rank * (int)blockDim.x + (int)threadIdx.x, stride = T * (int)blockDim.x;
    const int n = R.n;
    int total = 0;

    if (gid == 0) {
        atomicOr(&R.vis[R.q0 >> 5], 1u << (R.q0 & 31));
        R.f0[0] = R.q0;
        R.ctrl->fcnt[0] = 1;
    }
    if (!team_barrier(ts)) goto done;

    // ---- breadth-first levels: level L reads frontier L%2 (size fcnt[L%3]) and appends to
    //      frontier (L+1)%2 (size fcnt[(L+1)%3]); fcnt[(L+2)%3], last read at level L-1, is
    //      cleared for level L+1
    for (int level = 0, prev = 1 << 30;; ++level) {
        const int size = ld_volatile(&R.ctrl->fcnt[level % 3]);
        if (size == 0) break;
        const int budget = (size <= 4 && prev <= 4) ? kReachBudgetChain : kReachBudgetWide;
        prev = size;
        if (gid == 0) R.ctrl->fcnt[(level + 2) % 3] = 0;
        const int32_t* F = (level & 1) ? R.f1 : R.f0;
        int32_t* G = (level & 1) ? R.f0 : R.f1;
        int* gcnt = &R.ctrl->fcnt[(level + 1) % 3];
        for (int i = gid; i < size; i += stride) reach_expand(R, __ldcg(&F[i]), G, gcnt, budget);
        if (!team_barrier(ts)) goto done;
    }
    if (ld_volatile(&R.ctrl->status) != 0) goto done;

    // ---- order-preserving renumbering: CTA r owns bitmap words [w0, w1)
    {
        const int W = (n + 31) / 32;
        const int per = (W + T - 1) / T;
        const int w0 = min(W, rank * per), w1 = min(W, w0 + per);
        int local = 0;
        for (int w = w0 + (int)threadIdx.x; w < w1; w += blockDim.x)
            local += __popc(__ldcg(&R.vis[w]));
        local = cta_sum(local);
        if (threadIdx.x == 0) R.cta_sum[rank] = local;
        if (!team_barrier(ts)) goto done;
        int pre = 0;
        for (int r = threadIdx.x; r < rank; r += blockDim.x) pre += __ldcg(&R.cta_sum[r]);
        pre = cta_sum(pre);
        for (int base = w0; base < w1; base += blockDim.x) {
            const int w = base + (int)threadIdx.x;
            const uint32_t word = w < w1 ? __ldcg(&R.vis[w]) : 0u;
            int tile = 0;
            const int ex = cta_scan_count(__popc(word), &tile);
            if (w < w1) {
                for (int j = 0; j < 32; ++j) {
                    const int s = w * 32 + j;
                    if (s >= n) break;
                    R.newid[s] = ((word >> j) & 1u) ? pre + ex + __popc(word & ((1u << j) - 1u))
                                                   : -1;
                }
            }
            pre += tile;
        }
        if (rank == T - 1 && threadIdx.x == 0) total = pre;
        if (R.out_delta || R.out_accept) {
            if (!team_barrier(ts)) goto done;
            // ---- induced sub-DFA: reached state s becomes newid[s], successors likewise
            for (int s = w0 * 32 + (int)threadIdx.x; s < min(n, w1 * 32); s += blockDim.x) {
                const int id = __ldcg(&R.newid[s]);
                if (id < 0) continue;
                if (R.out_delta)
                    for (int a = 0; a < R.k; ++a)
                        R.out_delta[(int64_t)id * R.k + a] =
                            __ldcg(&R.newid[__ldg(&R.delta[(int64_t)s * R.k + a])]);
                if (R.out_accept && ((__ldg(&R.accept[s >> 5]) >> (s & 31)) & 1u))
                    atomicOr(&R.out_accept[id >> 5], 1u << (id & 31));
            }
        }
    }
done:
    if (threadIdx.x == 0 && rank == T - 1) {
        const int st = ld_volatile(&R.ctrl->status);
        if (R.count_out) *R.count_out = st ? -st : total;
        if (R.status_out) *R.status_out = st;
    }
}

struct QuotCtrl {
    unsigned long long bar;
    int status;
    int pad;
};

struct QuotJob {
    int32_t n, k, q0;
    const int32_t* delta;
    const uint32_t* accept;
    const int32_t* block;            // [n] class of every state (any ids in [0, n))
    const int32_t* newid;            // [n] or null: only states with newid >= 0 count
    const int32_t* prior_status[2];  // statuses of earlier stages (null = none)
    int32_t* rep;                    // [n] smallest counted member of each class id
    int32_t* newb;                   // [n] output number of each class id
    int32_t* cta_sum;                // [grid]
    int32_t* out_delta;              // [nstates*k]
    uint32_t* out_accept;            // [(n+31)/32], zeroed before the launch
    int32_t* nstates_out;            // device scalar: states of the quotient, or -status
    int32_t* q0_out;                 // device scalar or null
    int32_t* status_out;             // device scalar or null
    QuotCtrl* ctrl;
    int64_t timeout_ns;
};

__global__ void __launch_bounds__(kTeamThreads) quotient_kernel(QuotJob Q)
{
    TeamSync ts{&Q.ctrl->bar, &Q.ctrl->status, (unsigned long long)gridDim.x, 0ull,
                Q.timeout_ns};
    const int rank = blockIdx.x, T = gridDim.x;
    const int n = Q.n;
    const int chunk = ((n + T - 1) / T + 31) / 32 * 32;
    const int c0 = min(n, rank * chunk), c1 = min(n, c0 + chunk);
    int total = 0;

    if (rank == 0 && threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i)
            if (Q.prior_status[i]) {
                const int st = ld_volatile(Q.prior_status[i]);
                if (st != 0) atomicCAS(&Q.ctrl->status, 0, st);
            }
    }
    for (int s = c0 + (int)threadIdx.x; s < c1; s += blockDim.x) Q.rep[s] = 0x7fffffff;
    if (!team_barrier(ts)) goto done;

    // ---- representative of every class: its smallest counted member
    for (int s = c0 + (int)threadIdx.x; s < c1; s += blockDim.x) {
        if (Q.newid && __ldcg(&Q.newid[s]) < 0) continue;
        const int b = __ldg(&Q.block[s]);
        if ((unsigned)b >= (unsigned)n) {
            atomicCAS(&Q.ctrl->status, 0, (int)DFAMIN_EINVAL);
            continue;
        }
        atomicMin(&Q.rep[b], s);
    }
    if (!team_barrier(ts)) goto done;

    // ---- classes numbered in the order of their representatives
    {
        int local = 0;
        for (int s = c0 + (int)threadIdx.x; s < c1; s += blockDim.x) {
            const int b = __ldg(&Q.block[s]);
            local += (unsigned)b < (unsigned)n && __ldcg(&Q.rep[b]) == s;
        }
        local = cta_sum(local);
        if (threadIdx.x == 0) Q.cta_sum[rank] = local;
        if (!team_barrier(ts)) goto done;
        int pre = 0;
        for (int r = threadIdx.x; r < rank; r += blockDim.x) pre += __ldcg(&Q.cta_sum[r]);
        pre = cta_sum(pre);
        for (int base = c0; base < c1; base += blockDim.x) {
            const int s = base + (int)threadIdx.x;
            int b = -1;
            bool first = false;
            if (s < c1) {
                b = __ldg(&Q.block[s]);
                first = (unsigned)b < (unsigned)n && __ldcg(&Q.rep[b]) == s;
            }
            int tile = 0;
            const int ex = cta_scan_flag(first, &tile);
            if (first) Q.newb[b] = pre + ex;
            pre += tile;
        }
        if (rank == T - 1 && threadIdx.x == 0) total = pre;
    }
    if (!team_barrier(ts)) goto done;

    // ---- the quotient's transitions and accepting states, written by each representative
    for (int s = c0 + (int)threadIdx.x; s < c1; s += blockDim.x) {
        const int b = __ldg(&Q.block[s]);
        if ((unsigned)b >= (unsigned)n || __ldcg(&Q.rep[b]) != s) continue;
        const int id = __ldcg(&Q.newb[b]);
        for (int a = 0; a < Q.k; ++a) {
            const int t = __ldg(&Q.delta[(int64_t)s * Q.k + a]);
            if ((unsigned)t >= (unsigned)n) {
                atomicCAS(&Q.ctrl->status, 0, (int)DFAMIN_EINVAL);
                continue;
            }
            Q.out_delta[(int64_t)id * Q.k + a] = __ldcg(&Q.newb[__ldg(&Q.block[t])]);
        }
        if ((__ldg(&Q.accept[s >> 5]) >> (s & 31)) & 1u)
            atomicOr(&Q.out_accept[id >> 5], 1u << (id & 31));
    }
    if (rank == 0 && threadIdx.x == 0 && Q.q0_out)
        *Q.q0_out = __ldcg(&Q.newb[__ldg(&Q.block[Q.q0])]);
done:
    if (threadIdx.x == 0 && rank == T - 1) {
        const int st = ld_volatile(&Q.ctrl->status);
        if (Q.nstates_out) *Q.nstates_out = st ? -st : total;
        if (Q.status_out) *Q.status_out = st;
    }
}

}  // namespace dfamin_dev

using namespace dfamin_host;
using namespace dfamin_dev;

namespace {

struct ReachLayout {
    size_t ctrl, vis, f0, f1, cta, total;
};

ReachLayout reach_layout(int32_t n)
{
    const size_t A = 256;
    ReachLayout L{};
    size_t off = 0;
    L.ctrl = off; off = align_up(off + sizeof(ReachCtrl), A);
    L.vis = off; off = align_up(off + sizeof(uint32_t) * (size_t)((n + 31) / 32), A);
    L.f0 = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.f1 = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.cta = off; off = align_up(off + sizeof(int32_t) * kMaxCtas, A);
    L.total = off;
    return L;
}

struct QuotLayout {
    size_t ctrl, rep, newb, cta, total;
};

QuotLayout quot_layout(int32_t n)
{
    const size_t A = 256;
    QuotLayout L{};
    size_t off = 0;
    L.ctrl = off; off = align_up(off + sizeof(QuotCtrl), A);
    L.rep = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.newb = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.cta = off; off = align_up(off + sizeof(int32_t) * kMaxCtas, A);
    L.total = off;
    return L;
}

// Workspace of dfamin_minimal_dfa: [reach | newid | block | stage scalars | quotient |
// refinement workspace].
struct MinLayout {
    size_t reach, newid, block, scal, quot, refine, total;
};

MinLayout min_layout(int32_t n, size_t refine_bytes)
{
    const size_t A = 256;
    MinLayout L{};
    size_t off = 0;
    L.reach = off; off = align_up(off + reach_layout(n).total, A);
    L.newid = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.block = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    L.scal = off; off = align_up(off + sizeof(int32_t) * 8, A);
    L.quot = off; off = align_up(off + quot_layout(n).total, A);
    L.refine = off; off += refine_bytes;
    L.total = off;
    return L;
}

bool basic_args_ok(int32_t n, int32_t k, const int32_t* delta, const uint32_t* accept)
{
    if (n < 1 || n > (1 << 30) || k < 0 || (int64_t)n * (int64_t)k >= ((int64_t)1 << 40))
        return false;
    if ((k > 0 && !delta) || !accept) return false;
    return ((uintptr_t)delta & 3u) == 0 && ((uintptr_t)accept & 3u) == 0;
}

// Grid of a cooperative launch of `kernel`: all resident CTAs, fewer for small n.
dfamin_status coop_grid(const void* kernel, int32_t n, int* grid)
{
    int dev = 0, sms = 0;
    size_t smem_optin = 0;
    dfamin_status st = device_props(&dev, &sms, &smem_optin);
    if (st != DFAMIN_OK) return st;
    int per_sm = 0;
    st = kernel_ctas_per_sm(dev, kernel, kTeamThreads, 0, &per_sm);
    if (st != DFAMIN_OK) return st;
    int g = sms * per_sm;
    if (g > kMaxCtas) g = kMaxCtas;
    const int64_t want = ((int64_t)n + 2 * kTeamThreads - 1) / (2 * kTeamThreads);
    if (want < g) g = (int)(want > 0 ? want : 1);
    if (g < 1) return DFAMIN_ECUDA;
    *grid = g;
    return DFAMIN_OK;
}

dfamin_status launch_reach(int32_t n, int32_t k, const int32_t* delta, const uint32_t* accept,
                           int32_t q0, int32_t* out_newid, int32_t* out_delta,
                           uint32_t* out_accept, int32_t* count, int32_t* status, void* ws,
                           size_t ws_bytes, cudaStream_t stream)
{
    if (!basic_args_ok(n, k, delta, accept) || q0 < 0 || q0 >= n || !out_newid || !ws ||
        ((uintptr_t)ws & 255u) != 0 || ((uintptr_t)out_accept & 3u) != 0)
        return DFAMIN_EINVAL;
    const ReachLayout L = reach_layout(n);
    if (ws_bytes < L.total) return DFAMIN_ENOMEM;
    unsigned char* base = (unsigned char*)ws;
    ReachJob R{};
    R.n = n; R.k = k; R.q0 = q0;
    R.delta = delta; R.accept = accept;
    R.vis = (uint32_t*)(base + L.vis);
    R.f0 = (int32_t*)(base + L.f0);
    R.f1 = (int32_t*)(base + L.f1);
    R.cta_sum = (int32_t*)(base + L.cta);
    R.newid = out_newid;
    R.out_delta = k > 0 ? out_delta : nullptr;
    R.out_accept = out_accept;
    R.count_out = count;
    R.status_out = status;
    R.ctrl = (ReachCtrl*)(base + L.ctrl);
    R.timeout_ns = kBarrierTimeoutNs;
    if (!cuda_ok(cudaMemsetAsync(base, 0, L.f0, stream), "cudaMemsetAsync(reach)"))
        return DFAMIN_ECUDA;
    if (out_accept &&
        !cuda_ok(cudaMemsetAsync(out_accept, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32),
                                 stream),
                 "cudaMemsetAsync(out_accept)"))
        return DFAMIN_ECUDA;
    int grid = 0;
    const dfamin_status st = coop_grid((const void*)reach_kernel, n, &grid);
    if (st != DFAMIN_OK) return st;
    void* args[] = {&R};
    if (!cuda_ok(cudaLaunchCooperativeKernel((const void*)reach_kernel, dim3(grid),
                                             dim3(kTeamThreads), args, 0, stream),
                 "reach_kernel cooperative launch"))
        return DFAMIN_ECUDA;
    return DFAMIN_OK;
}

dfamin_status launch_quotient(int32_t n, int32_t k, const int32_t* delta, const uint32_t* accept,
                              const int32_t* block, int32_t q0, const int32_t* newid,
                              const int32_t* prior0, const int32_t* prior1, int32_t* out_delta,
                              uint32_t* out_accept, int32_t* nstates, int32_t* out_q0,
                              int32_t* status, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!basic_args_ok(n, k, delta, accept) || q0 < 0 || q0 >= n || !block ||
        (k > 0 && !out_delta) || !out_accept || !nstates || !ws ||
        ((uintptr_t)ws & 255u) != 0 || ((uintptr_t)out_accept & 3u) != 0)
        return DFAMIN_EINVAL;
    const QuotLayout L = quot_layout(n);
    if (ws_bytes < L.total) return DFAMIN_ENOMEM;
    unsigned char* base = (unsigned char*)ws;
    QuotJob Q{};
    Q.n = n; Q.k = k; Q.q0 = q0;
    Q.delta = delta; Q.accept = accept; Q.block = block; Q.newid = newid;
    Q.prior_status[0] = prior0;
    Q.prior_status[1] = prior1;
    Q.rep = (int32_t*)(base + L.rep);
    Q.newb = (int32_t*)(base + L.newb);
    Q.cta_sum = (int32_t*)(base + L.cta);
    Q.out_delta = out_delta;
    Q.out_accept = out_accept;
    Q.nstates_out = nstates;
    Q.q0_out = out_q0;
    Q.status_out = status;
    Q.ctrl = (QuotCtrl*)(base + L.ctrl);
    Q.timeout_ns = kBarrierTimeoutNs;
    if (!cuda_ok(cudaMemsetAsync(base, 0, sizeof(QuotCtrl), stream), "cudaMemsetAsync(quot)"))
        return DFAMIN_ECUDA;
    if (!cuda_ok(cudaMemsetAsync(out_accept, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32),
                                 stream),
                 "cudaMemsetAsync(out_accept)"))
        return DFAMIN_ECUDA;
    int grid = 0;
    const dfamin_status st = coop_grid((const void*)quotient_kernel, n, &grid);
    if (st != DFAMIN_OK) return st;
    void* args[] = {&Q};
    if (!cuda_ok(cudaLaunchCooperativeKernel((const void*)quotient_kernel, dim3(grid),
                                             dim3(kTeamThreads), args, 0, stream),
                 "quotient_kernel cooperative launch"))
        return DFAMIN_ECUDA;
    return DFAMIN_OK;
}

}  // namespace

DFAMIN_API dfamin_status dfamin_reach_workspace_size(int32_t n, size_t* bytes)
{
    if (n < 1 || n > (1 << 30) || !bytes) return DFAMIN_EINVAL;
    *bytes = reach_layout(n).total;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_reachable(int32_t n, int32_t k, const int32_t* delta,
                                          const uint32_t* accept, int32_t q0,
                                          int32_t* out_newid, int32_t* out_delta,
                                          uint32_t* out_accept, int32_t* count, int32_t* status,
                                          void* workspace, size_t workspace_bytes,
                                          dfamin_stream_t stream)
{
    return launch_reach(n, k, delta, accept, q0, out_newid, out_delta, out_accept, count, status,
                        workspace, workspace_bytes, (cudaStream_t)stream);
}

DFAMIN_API dfamin_status dfamin_quotient_workspace_size(int32_t n, size_t* bytes)
{
    if (n < 1 || n > (1 << 30) || !bytes) return DFAMIN_EINVAL;
    *bytes = quot_layout(n).total;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_quotient(int32_t n, int32_t k, const int32_t* delta,
                                         const uint32_t* accept, const int32_t* block,
                                         int32_t q0, const int32_t* newid, int32_t* out_delta,
                                         uint32_t* out_accept, int32_t* nstates, int32_t* out_q0,
                                         int32_t* status, void* workspace,
                                         size_t workspace_bytes, dfamin_stream_t stream)
{
    return launch_quotient(n, k, delta, accept, block, q0, newid, nullptr, nullptr, out_delta,
                           out_accept, nstates, out_q0, status, workspace, workspace_bytes,
                           (cudaStream_t)stream);
}

DFAMIN_API dfamin_status dfamin_minimal_dfa_workspace_size(int32_t n, int32_t k,
                                                           const dfamin_options* opt,
                                                           size_t* bytes)
{
    if (!bytes) return DFAMIN_EINVAL;
    size_t refine = 0;
    const dfamin_status st = dfamin_workspace_size(n, k, opt, &refine);
    if (st != DFAMIN_OK) return st;
    *bytes = min_layout(n, refine).total;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_minimal_dfa(int32_t n, int32_t k, const int32_t* delta,
                                            const uint32_t* accept, int32_t q0,
                                            const dfamin_options* opt, int32_t* out_delta,
                                            uint32_t* out_accept, int32_t* out_scalars,
                                            void* workspace, size_t workspace_bytes,
                                            dfamin_stream_t stream)
{
    if (!out_scalars || !workspace || ((uintptr_t)workspace & 255u) != 0) return DFAMIN_EINVAL;
    size_t refine = 0;
    dfamin_status st = dfamin_workspace_size(n, k, opt, &refine);
    if (st != DFAMIN_OK) return st;
    const MinLayout L = min_layout(n, refine);
    if (workspace_bytes < L.total) return DFAMIN_ENOMEM;
    if (!basic_args_ok(n, k, delta, accept) || q0 < 0 || q0 >= n || (k > 0 && !out_delta) ||
        !out_accept)
        return DFAMIN_EINVAL;
    unsigned char* base = (unsigned char*)workspace;
    int32_t* newid = (int32_t*)(base + L.newid);
    int32_t* block = (int32_t*)(base + L.block);
    int32_t* scal = (int32_t*)(base + L.scal);   // [0] nblocks [1] reach status [2] refine status
    cudaStream_t s = (cudaStream_t)stream;
    st = launch_reach(n, k, delta, accept, q0, newid, nullptr, nullptr, out_scalars + 2,
                      scal + 1, base + L.reach, L.newid - L.reach, s);
    if (st != DFAMIN_OK) return st;
    st = dfamin_minimize_ex(n, k, delta, accept, block, scal, opt, base + L.refine, refine,
                            out_scalars + 3, scal + 2, stream);
    if (st != DFAMIN_OK) return st;
    return launch_quotient(n, k, delta, accept, block, q0, newid, scal + 1, scal + 2, out_delta,
                           out_accept, out_scalars, out_scalars + 1, out_scalars + 4,
                           base + L.quot, L.refine - L.quot, s);
}

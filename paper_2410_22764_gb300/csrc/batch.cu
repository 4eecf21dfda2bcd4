// dfamin batch entry points: thousands of DFAs of uneven sizes minimized in ONE persistent
// cooperative launch (capturable in a CUDA graph).
//
// Every DFA is refined exactly as by dfamin_minimize_ex (refine.cuh): signature rounds of
// Alg. sortPR (Sec. 3.3), optionally on the closed DFA of Alg. transPR (Sec. 3.4).  What this
// file adds is the scheduling:
//   * a plan (host metadata only) sorts the DFAs by decreasing work and gives each a team size:
//     one CTA in shared memory for small DFAs, otherwise ceil(n / team_states) CTAs (capped by
//     the grid);
//   * the team sizes are laid out as consecutive "tickets"; every CTA of the grid repeatedly
//     takes the next ticket from one counter and becomes member (ticket - first ticket) of that
//     DFA's team.  Tickets are taken in order, so every team whose last ticket has been taken is
//     complete and makes progress; the team waiting for members is the one with the newest
//     tickets, and its members arrive as soon as earlier (larger) DFAs finish;
//   * team members meet at bounded barriers on the DFA's own control block, exactly as the
//     single-DFA kernel's CTAs do.

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "dfamin.h"
#include "refine.cuh"
#include "host_common.h"

namespace dfamin_dev {

constexpr int64_t kBatchBarrierTimeoutNs = 30000000000ll;  // 30 s: a team may wait for members

struct BatchDesc {             // one DFA, in ticket order
    int64_t state_off;         // its first state in the concatenated state space
    int64_t delta_off;         // its first entry in the concatenated delta
    int64_t region;            // byte offset of its arrays in the workspace
    int64_t ticket0;           // first ticket of its team
    int32_t n, k;
    int32_t team;              // CTAs
    int32_t small;             // 1: one CTA, shared-memory path
    int32_t index;             // position in the caller's per-DFA arrays
    uint32_t small_cap;        // shared table capacity (small path)
    uint32_t cap;              // global table capacity (team path)
    int32_t levels, sig_stride, max_passes;
    int32_t cl_cols;           // closure columns its region holds
    int32_t cta_base;          // first entry of its per-CTA counts
    int32_t nonid_base;        // first entry of its identity-letter flags
    int32_t pat_base;          // first entry of its round-1 pattern minima, -1 = none
    int64_t o_block, o_lst_s, o_lst_slot, o_lst_rst, o_lead, o_lead_slot, o_stg, o_table, o_sig,
        o_cl, o_cl_letter, o_naive, o_spl, o_cln;
};

struct BatchArgs {
    const BatchDesc* desc;
    int32_t count;
    int64_t tickets;
    const int32_t* delta;
    const uint32_t* accept;
    int32_t* out_block;
    int32_t* nblocks;
    int32_t* passes;
    int32_t* status;
    unsigned char* ws;
    unsigned long long* ticket;    // zeroed per launch
    Ctrl* ctrl;                    // [count], zeroed per launch, indexed by the caller's index
    int32_t* nonid;                // zeroed per launch
    int32_t* pat;                  // zeroed per launch: round-1 pattern minima of team DFAs
    int32_t* cta_cnt;
    uint32_t flags;
    int32_t algo;
    int64_t timeout_ns;            // bound on every team barrier wait
};

__device__ Job batch_job(const BatchArgs& A, const BatchDesc& D)
{
    Job J{};
    J.n = D.n;
    J.k = D.k;
    J.delta = A.delta + D.delta_off;
    J.accept = A.accept;
    J.acc_off = D.state_off;
    J.out_block = A.out_block + D.state_off;
    J.nblocks_out = A.nblocks + D.index;
    J.passes_out = A.passes ? A.passes + D.index : nullptr;
    J.status_out = A.status ? A.status + D.index : nullptr;
    J.ctrl = A.ctrl + D.index;
    J.cta_cnt = A.cta_cnt + D.cta_base;
    J.nonid = A.nonid + D.nonid_base;
    J.pat_rev = D.pat_base >= 0 ? A.pat + D.pat_base : nullptr;
    unsigned char* r = A.ws + D.region;
    J.cl_letter = (int32_t*)(r + D.o_cl_letter);
    J.block = (int32_t*)(r + D.o_block);
    J.lst_s = (int32_t*)(r + D.o_lst_s);
    J.lst_slot = (uint32_t*)(r + D.o_lst_slot);
    J.lst_rst = (uint32_t*)(r + D.o_lst_rst);
    J.lead = (int32_t*)(r + D.o_lead);
    J.lead_slot = (uint32_t*)(r + D.o_lead_slot);
    J.stg = (int32_t*)(r + D.o_stg);
    J.naive_new = (int32_t*)(r + D.o_naive);
    J.spl = (int32_t*)(r + D.o_spl);
    J.cln = (int32_t*)(r + D.o_cln);
    J.algo = A.algo;
    J.table = (unsigned long long*)(r + D.o_table);
    J.mask = D.cap - 1;
    J.sig = (int32_t*)(r + D.o_sig);
    J.sig_stride = D.sig_stride;
    J.cl = (int32_t*)(r + D.o_cl);
    J.levels = D.levels;
    J.cl_cols = D.cl_cols;
    J.max_passes = D.max_passes;
    J.flags = A.flags;
    J.timeout_ns = A.timeout_ns;
    J.trace = nullptr;
    return J;
}

// Separate (not inlined) functions: each alphabet size gets its own register allocation.
template <int KC>
__device__ __noinline__ void run_team(const Job& J, int rank, int T)
{
    TeamSync ts{&J.ctrl->bar, &J.ctrl->status, (unsigned long long)T, 0ull, J.timeout_ns};
    team_minimize<KC>(J, rank, T, ts);
}

__device__ __noinline__ void run_small(const Job& J, uint32_t cap) { small_minimize(J, cap); }

// The batch kernel, compiled for MINB resident CTAs per SM: 3 (80 registers a thread) by
// default, 4 (64 registers, more spills) with DFAMIN_FLAG_BATCH_FOUR_CTAS.  A tuning knob only.
template <int MINB>
__global__ void __launch_bounds__(kTeamThreads, MINB) batch_kernel(BatchArgs A)
{
    __shared__ long long s_ticket;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_ticket = (long long)atomicAdd(A.ticket, 1ull);
        __syncthreads();
        const long long t = s_ticket;
        if (t >= A.tickets) return;
        int lo = 0, hi = A.count - 1;                 // last DFA whose first ticket <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.desc[mid].ticket0 <= t) lo = mid; else hi = mid - 1;
        }
        const BatchDesc D = A.desc[lo];
        const Job J = batch_job(A, D);
        const int rank = (int)(t - D.ticket0);
        if (D.small) {
            run_small(J, D.small_cap);
            continue;
        }
        // compile-time alphabets need delta aligned for their vector row loads
        const int need = (D.k % 4 == 0) ? 16 : ((D.k % 2 == 0) ? 8 : 4);
        const bool aligned = ((uintptr_t)J.delta % need) == 0;
        if (D.levels == 1 && aligned) {
            switch (D.k) {
            case 1: run_team<1>(J, rank, D.team); continue;
            case 2: run_team<2>(J, rank, D.team); continue;
            case 3: run_team<3>(J, rank, D.team); continue;
            case 4: run_team<4>(J, rank, D.team); continue;
            case 5: run_team<5>(J, rank, D.team); continue;
            case 6: run_team<6>(J, rank, D.team); continue;
            case 7: run_team<7>(J, rank, D.team); continue;
            case 8: run_team<8>(J, rank, D.team); continue;
            default: break;
            }
        }
        run_team<0>(J, rank, D.team);
    }
}

}  // namespace dfamin_dev

using namespace dfamin_host;
using namespace dfamin_dev;

struct dfamin_batch_plan_s {
    int dev = 0;
    int32_t count = 0;
    dfamin_options opt{};
    std::vector<BatchDesc> desc;   // ticket order
    BatchDesc* d_desc = nullptr;   // device copy, owned
    cudaEvent_t last_launch = nullptr;  // recorded on the stream of every uncaptured launch
    bool recorded = false;              // last_launch has been recorded at least once
    int64_t tickets = 0;
    int grid = 0;
    size_t dsmem = 0;
    size_t off_ctrl = 0, off_nonid = 0, off_pat = 0, zero_end = 0, off_cta = 0, ws_bytes = 0;
    int64_t total_states = 0, total_delta = 0;
};

namespace {

constexpr int kBatchSmallDefault = 2048;     // n up to this: one CTA in shared memory

const void* batch_kernel_for(uint32_t flags)
{
    return (flags & DFAMIN_FLAG_BATCH_FOUR_CTAS) ? (const void*)batch_kernel<4>
                                                 : (const void*)batch_kernel<3>;
}

// Plans keep their descriptor table in stream-ordered memory (cudaMallocAsync / cudaFreeAsync
// on a library stream per device), so that creating or destroying a plan never waits for work
// running on other streams.
std::map<int, cudaStream_t> g_plan_streams;

dfamin_status plan_stream(int dev, cudaStream_t* out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_plan_streams.find(dev);
    if (it == g_plan_streams.end()) {
        cudaStream_t s = nullptr;
        if (!cuda_ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate"))
            return DFAMIN_ECUDA;
        it = g_plan_streams.emplace(dev, s).first;
    }
    *out = it->second;
    return DFAMIN_OK;
}
constexpr int kBatchTeamStatesDefault = 16384;

size_t cache_bytes_for(int k, bool closure)
{
    if (closure) return 0;
    switch (k) {
    case 1: return sizeof(CacheOf<1>::type);
    case 2: return sizeof(CacheOf<2>::type);
    case 3: return sizeof(CacheOf<3>::type);
    case 4: return sizeof(CacheOf<4>::type);
    case 5: return sizeof(CacheOf<5>::type);
    case 6: return sizeof(CacheOf<6>::type);
    case 7: return sizeof(CacheOf<7>::type);
    case 8: return sizeof(CacheOf<8>::type);
    default: return 0;
    }
}

}  // namespace

namespace {

// The host schedule of a batch: ticket order, team sizes, workspace layout, descriptors.
dfamin_status build_schedule(int32_t count, const int64_t* state_off, const int32_t* k,
                             const dfamin_options* opt, dfamin_batch_plan_s* P)
{
    if (count < 1 || !state_off || !k) return DFAMIN_EINVAL;
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    if (state_off[0] != 0) return DFAMIN_EINVAL;
    int64_t total_delta = 0;
    for (int32_t i = 0; i < count; ++i) {
        const int64_t n = state_off[i + 1] - state_off[i];
        if (n < 1 || n > (1 << 30) || k[i] < 0) return DFAMIN_EINVAL;
        total_delta += n * (int64_t)k[i];
        if (total_delta >= ((int64_t)1 << 40)) return DFAMIN_EINVAL;
    }
    int dev = 0, sms = 0;
    size_t smem_optin = 0;
    st = device_props(&dev, &sms, &smem_optin);
    if (st != DFAMIN_OK) return st;

    const bool closure = o.closure == DFAMIN_CLOSURE_ON;
    const int small_limit = std::min(o.smem_states > 0 ? o.smem_states : kBatchSmallDefault,
                                     kSmallMaxStates);
    const int team_states = o.team_states > 0 ? o.team_states : kBatchTeamStatesDefault;

    // dynamic shared memory: the largest small DFA's tables and the largest group cache
    size_t dsmem = 0;
    for (int32_t i = 0; i < count; ++i) {
        const int64_t n = state_off[i + 1] - state_off[i];
        if (n <= small_limit && o.algorithm == DFAMIN_ALG_SIGNATURE)
            dsmem = std::max(dsmem, small_smem_bytes((int32_t)n, nullptr));
        else dsmem = std::max(dsmem, cache_bytes_for(k[i], closure));
    }
    if (dsmem + 2048 > smem_optin) return DFAMIN_EINVAL;
    int per_sm = 0;
    st = kernel_ctas_per_sm(dev, batch_kernel_for(o.flags), kTeamThreads, dsmem, &per_sm);
    if (st != DFAMIN_OK) return st;
    int grid_max = std::min(sms * per_sm, kMaxCtas);
    if (o.ctas > 0) grid_max = std::min(grid_max, o.ctas);
    if (grid_max < 1) return DFAMIN_ECUDA;

    P->dev = dev;
    P->count = count;
    P->opt = o;
    P->total_states = state_off[count];
    P->total_delta = total_delta;
    P->dsmem = dsmem;

    // order: decreasing work, so large teams form first while every CTA is free
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int64_t wa = (state_off[a + 1] - state_off[a]) * (int64_t)(k[a] + 1);
        const int64_t wb = (state_off[b + 1] - state_off[b]) * (int64_t)(k[b] + 1);
        return wa > wb;
    });

    const size_t A = 256;
    size_t off = 256;                                // [0, 256): ticket counter
    P->off_ctrl = off; off = align_up(off + sizeof(Ctrl) * (size_t)count, A);
    int64_t ksum = 0, team_sum = 0, patsum = 0;
    P->desc.resize(count);
    for (int32_t j = 0; j < count; ++j) {
        const int32_t i = order[j];
        BatchDesc& D = P->desc[j];
        memset(&D, 0, sizeof(D));
        D.index = i;
        D.n = (int32_t)(state_off[i + 1] - state_off[i]);
        D.k = k[i];
        D.state_off = state_off[i];
        D.small = (D.n <= small_limit && o.algorithm == DFAMIN_ALG_SIGNATURE) ? 1 : 0;
        D.team = D.small ? 1
                         : (int32_t)std::min<int64_t>(
                               std::max<int64_t>(1, ((int64_t)D.n + team_states - 1) / team_states),
                               grid_max);
        D.ticket0 = team_sum;
        team_sum += D.team;
        D.cta_base = (int32_t)(team_sum - D.team);
        D.nonid_base = (int32_t)ksum;
        ksum += std::max(1, D.k);
        D.pat_base = -1;
        if (!D.small && !closure && D.k >= 1 && D.k <= kPatMaxK) {
            D.pat_base = (int32_t)patsum;
            patsum += 1 << (D.k + 1);
        }
        D.max_passes = o.max_passes > 0 ? o.max_passes : (D.n < 0x7fffffff ? D.n + 1 : D.n);
        if (D.small) small_smem_bytes(D.n, &D.small_cap);
    }
    // delta offsets in the caller's (original) order
    {
        std::vector<int64_t> doff(count + 1, 0);
        for (int32_t i = 0; i < count; ++i)
            doff[i + 1] = doff[i] + (state_off[i + 1] - state_off[i]) * (int64_t)k[i];
        for (auto& D : P->desc) D.delta_off = doff[D.index];
    }
    P->off_nonid = off; off = align_up(off + sizeof(int32_t) * (size_t)ksum, A);
    P->off_pat = off; off = align_up(off + sizeof(int32_t) * (size_t)std::max<int64_t>(1, patsum), A);
    P->zero_end = off;
    P->off_cta = off; off = align_up(off + sizeof(int32_t) * (size_t)team_sum, A);
    for (auto& D : P->desc) {
        const DfaLayout L = make_dfa_layout(D.n, D.k, closure, !D.small, o.closure_columns);
        D.region = (int64_t)off;
        D.cap = L.cap;
        D.levels = L.levels;
        D.cl_cols = L.cols;
        D.sig_stride = L.sig_stride;
        D.o_block = L.block; D.o_lst_s = L.lst_s; D.o_lst_slot = L.lst_slot;
        D.o_lst_rst = L.lst_rst; D.o_lead = L.lead; D.o_lead_slot = L.lead_slot; D.o_stg = L.stg;
        D.o_table = L.table; D.o_sig = L.sig; D.o_cl = L.cl; D.o_cl_letter = L.cl_letter;
        D.o_naive = L.naive_new;
        D.o_spl = L.spl;
        D.o_cln = L.cln;
        off = align_up(off + L.total, A);
    }
    P->ws_bytes = off;
    P->tickets = team_sum;
    P->grid = (int)std::min<int64_t>(grid_max, team_sum);

    return DFAMIN_OK;
}

}  // namespace

DFAMIN_API dfamin_status dfamin_batch_plan_create(int32_t count, const int64_t* state_off,
                                                  const int32_t* k, const dfamin_options* opt,
                                                  dfamin_batch_plan* plan_out)
{
    if (!plan_out) return DFAMIN_EINVAL;
    *plan_out = nullptr;
    auto* P = new dfamin_batch_plan_s;
    dfamin_status st = build_schedule(count, state_off, k, opt, P);
    if (st != DFAMIN_OK) {
        delete P;
        return st;
    }
    const int dev = P->dev;
    cudaStream_t ps = nullptr;
    st = plan_stream(dev, &ps);
    if (st != DFAMIN_OK) {
        delete P;
        return st;
    }
    if (!cuda_ok(cudaEventCreateWithFlags(&P->last_launch, cudaEventDisableTiming),
                 "cudaEventCreate(plan)")) {
        delete P;
        return DFAMIN_ECUDA;
    }
    if (!cuda_ok(cudaMallocAsync((void**)&P->d_desc, sizeof(BatchDesc) * (size_t)count, ps),
                 "cudaMallocAsync(plan)")) {
        cudaEventDestroy(P->last_launch);
        delete P;
        return DFAMIN_ENOMEM;
    }
    if (!cuda_ok(cudaMemcpyAsync(P->d_desc, P->desc.data(), sizeof(BatchDesc) * (size_t)count,
                                 cudaMemcpyHostToDevice, ps),
                 "cudaMemcpyAsync(plan)") ||
        !cuda_ok(cudaStreamSynchronize(ps), "cudaStreamSynchronize(plan)")) {
        cudaFreeAsync(P->d_desc, ps);
        cudaEventDestroy(P->last_launch);
        delete P;
        return DFAMIN_ECUDA;
    }
    *plan_out = P;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_batch_plan_destroy(dfamin_batch_plan plan)
{
    if (!plan) return DFAMIN_EINVAL;
    if (plan->d_desc) {
        // the table is freed in stream order after the last launch that used the plan (even if
        // that launch is still running), without blocking the host
        cudaStream_t ps = nullptr;
        if (plan_stream(plan->dev, &ps) == DFAMIN_OK) {
            if (plan->recorded) cudaStreamWaitEvent(ps, plan->last_launch, 0);
            cudaFreeAsync(plan->d_desc, ps);
        }
    }
    if (plan->last_launch) cudaEventDestroy(plan->last_launch);
    delete plan;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_batch_workspace_size(dfamin_batch_plan plan, size_t* bytes)
{
    if (!plan || !bytes) return DFAMIN_EINVAL;
    *bytes = plan->ws_bytes;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_batch_plan_info(dfamin_batch_plan plan, int32_t* grid,
                                                int64_t* tickets, int64_t* states,
                                                int64_t* transitions)
{
    if (!plan) return DFAMIN_EINVAL;
    if (grid) *grid = plan->grid;
    if (tickets) *tickets = plan->tickets;
    if (states) *states = plan->total_states;
    if (transitions) *transitions = plan->total_delta;
    return DFAMIN_OK;
}

namespace {

// One launch of a scheduled batch: descriptors at d_desc (device), workspace at base.
dfamin_status launch_batch(const dfamin_batch_plan_s& P, const BatchDesc* d_desc,
                           unsigned char* base, const int32_t* delta, const uint32_t* accept,
                           int32_t* out_block, int32_t* nblocks, int32_t* passes,
                           int32_t* status, cudaStream_t stream)
{
    if (!cuda_ok(cudaMemsetAsync(base, 0, P.zero_end, stream), "cudaMemsetAsync(batch control)"))
        return DFAMIN_ECUDA;
    BatchArgs A{};
    A.desc = d_desc;
    A.count = P.count;
    A.tickets = P.tickets;
    A.delta = delta;
    A.accept = accept;
    A.out_block = out_block;
    A.nblocks = nblocks;
    A.passes = passes;
    A.status = status;
    A.ws = base;
    A.ticket = (unsigned long long*)base;
    A.ctrl = (Ctrl*)(base + P.off_ctrl);
    A.nonid = (int32_t*)(base + P.off_nonid);
    A.pat = (int32_t*)(base + P.off_pat);
    A.cta_cnt = (int32_t*)(base + P.off_cta);
    A.flags = P.opt.flags & ~DFAMIN_FLAG_TRACE;
    A.algo = P.opt.algorithm;
    A.timeout_ns = P.opt.barrier_timeout_us > 0 ? 1000ll * P.opt.barrier_timeout_us
                                                : kBatchBarrierTimeoutNs;
    void* args[] = {&A};
    if (!cuda_ok(cudaLaunchCooperativeKernel(batch_kernel_for(P.opt.flags), dim3(P.grid),
                                             dim3(kTeamThreads), args, P.dsmem, stream),
                 "batch_kernel cooperative launch"))
        return DFAMIN_ECUDA;
    return DFAMIN_OK;
}

dfamin_status check_batch_args(const dfamin_batch_plan_s& P, const int32_t* delta,
                               const uint32_t* accept, int32_t* out_block, int32_t* nblocks,
                               void* workspace)
{
    if (!accept || !out_block || !nblocks || !workspace) return DFAMIN_EINVAL;
    if (P.total_delta > 0 && !delta) return DFAMIN_EINVAL;
    if (((uintptr_t)workspace & 255u) != 0 || ((uintptr_t)delta & 3u) != 0 ||
        ((uintptr_t)accept & 3u) != 0)
        return DFAMIN_EINVAL;
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return DFAMIN_ECUDA;
    if (dev != P.dev) return DFAMIN_EINVAL;
    return DFAMIN_OK;
}

}  // namespace

DFAMIN_API dfamin_status dfamin_batch_plan_run(dfamin_batch_plan plan, const int32_t* delta,
                                               const uint32_t* accept, int32_t* out_block,
                                               int32_t* nblocks, int32_t* passes,
                                               int32_t* status, void* workspace,
                                               size_t workspace_bytes, dfamin_stream_t stream)
{
    if (!plan) return DFAMIN_EINVAL;
    dfamin_status st = check_batch_args(*plan, delta, accept, out_block, nblocks, workspace);
    if (st != DFAMIN_OK) return st;
    if (workspace_bytes < plan->ws_bytes) return DFAMIN_ENOMEM;
    st = launch_batch(*plan, plan->d_desc, (unsigned char*)workspace, delta, accept, out_block,
                      nblocks, passes, status, (cudaStream_t)stream);
    if (st != DFAMIN_OK) return st;
    // outside stream capture the launch is marked so that the plan's release waits for it; a
    // launch captured into a graph cannot be waited on from outside, and the caller keeps the
    // plan alive while the graph may be replayed
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!cuda_ok(cudaStreamIsCapturing((cudaStream_t)stream, &cap), "cudaStreamIsCapturing"))
        return DFAMIN_ECUDA;
    if (cap == cudaStreamCaptureStatusNone) {
        if (!cuda_ok(cudaEventRecord(plan->last_launch, (cudaStream_t)stream),
                     "cudaEventRecord(plan)"))
            return DFAMIN_ECUDA;
        plan->recorded = true;
    }
    return DFAMIN_OK;
}

// ------------------------------------------------------------------------------------------
// One-shot batch: the schedule is computed on the host for this call and its descriptor table
// is copied into the head of the caller's workspace, so nothing is allocated.
// ------------------------------------------------------------------------------------------
namespace {

dfamin_status one_shot_layout(int32_t num_dfas, const int64_t* state_off, const int32_t* k,
                              const int64_t* delta_off, const dfamin_options* opt,
                              dfamin_batch_plan_s* P, size_t* desc_bytes)
{
    dfamin_status st = build_schedule(num_dfas, state_off, k, opt, P);
    if (st != DFAMIN_OK) return st;
    if (delta_off) {
        if (delta_off[0] != 0) return DFAMIN_EINVAL;
        for (int32_t i = 0; i < num_dfas; ++i)
            if (delta_off[i + 1] - delta_off[i] != (state_off[i + 1] - state_off[i]) * (int64_t)k[i])
                return DFAMIN_EINVAL;
    }
    *desc_bytes = align_up(sizeof(BatchDesc) * (size_t)num_dfas, 256);
    return DFAMIN_OK;
}

}  // namespace

DFAMIN_API dfamin_status dfamin_minimize_batch_workspace_size(int32_t num_dfas,
                                                              const int64_t* state_off,
                                                              const int32_t* k,
                                                              const dfamin_options* opt,
                                                              size_t* bytes)
{
    if (!bytes) return DFAMIN_EINVAL;
    dfamin_batch_plan_s P;
    size_t desc_bytes = 0;
    const dfamin_status st = one_shot_layout(num_dfas, state_off, k, nullptr, opt, &P, &desc_bytes);
    if (st != DFAMIN_OK) return st;
    *bytes = desc_bytes + P.ws_bytes;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_minimize_batch(int32_t num_dfas, const int64_t* state_off,
                                               const int32_t* k, const int64_t* delta_off,
                                               const int32_t* delta, const uint32_t* accept,
                                               int32_t* out_block, int32_t* nblocks,
                                               const dfamin_options* opt, void* workspace,
                                               size_t workspace_bytes, int32_t* status,
                                               dfamin_stream_t stream)
{
    // the descriptor table is copied from host memory that lives only during this call, so a
    // captured copy would replay from freed memory: refuse capture (plans are the capturable form)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!cuda_ok(cudaStreamIsCapturing((cudaStream_t)stream, &cap), "cudaStreamIsCapturing"))
        return DFAMIN_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "dfamin_minimize_batch: the stream is capturing; use a batch plan in graphs");
        return DFAMIN_EINVAL;
    }
    dfamin_batch_plan_s P;
    size_t desc_bytes = 0;
    dfamin_status st = one_shot_layout(num_dfas, state_off, k, delta_off, opt, &P, &desc_bytes);
    if (st != DFAMIN_OK) return st;
    st = check_batch_args(P, delta, accept, out_block, nblocks, workspace);
    if (st != DFAMIN_OK) return st;
    if (workspace_bytes < desc_bytes + P.ws_bytes) return DFAMIN_ENOMEM;
    unsigned char* base = (unsigned char*)workspace;
    // pageable source: the call returns once the table is staged, so the host vector may go
    if (!cuda_ok(cudaMemcpyAsync(base, P.desc.data(), sizeof(BatchDesc) * (size_t)num_dfas,
                                 cudaMemcpyHostToDevice, (cudaStream_t)stream),
                 "cudaMemcpyAsync(batch table)"))
        return DFAMIN_ECUDA;
    return launch_batch(P, reinterpret_cast<const BatchDesc*>(base), base + desc_bytes, delta,
                        accept, out_block, nblocks, nullptr, status, (cudaStream_t)stream);
}

// dfamin: single-DFA entry points (dfamin_minimize, _ex, _static) on GB300 (sm_103a).
// The refinement itself is in refine.cuh; the shared host helpers in host_common.h.

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "dfamin.h"
#include "refine.cuh"
#include "host_common.h"

namespace dfamin_dev {

// CTA shape of the single-DFA team kernel: 512 threads, two CTAs (64 registers a thread) per SM
// for k <= 5 and the runtime width; 256 threads, three CTAs (80 registers) for k = 6..8.  With
// half as many CTAs as 256-thread ones the team's barriers gather half the arrivals (measured:
// plain path rounds 17.6 -> 16.2 us, the inflated n = 10^7 DFA 0.940 -> 0.929 ms).
template <int KC>
struct TeamShape {
    static constexpr int threads = (KC >= 6) ? 256 : 512;
    static constexpr int min_ctas = (KC >= 6) ? 3 : 2;
};

template <int KC>
__global__ void __launch_bounds__(TeamShape<KC>::threads, TeamShape<KC>::min_ctas) team_kernel(Job J)
{
    TeamSync ts{&J.ctrl->bar, &J.ctrl->status, (unsigned long long)gridDim.x, 0ull, J.timeout_ns};
    team_minimize<KC>(J, blockIdx.x, gridDim.x, ts);
}

__global__ void __launch_bounds__(kThreads) small_kernel(Job J, uint32_t cap)
{
    small_minimize(J, cap);
}

__global__ void __launch_bounds__(kMediumThreads, 1) medium_kernel(Job J)
{
    medium_minimize(J);
}

}  // namespace dfamin_dev

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
namespace dfamin_host {

std::mutex g_mu;
thread_local char g_last_error[256] = "";

bool cuda_ok(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return true;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", what, cudaGetErrorString(e),
             (int)e);
    return false;
}

namespace {
struct Props {
    int sms = 0;
    size_t smem_optin = 0;
};
std::map<int, Props> g_props;
std::map<std::pair<std::pair<int, const void*>, std::pair<int, size_t>>, int> g_occ;
std::map<std::pair<int, const void*>, int> g_attr_set;   // (device, kernel) -> dynamic smem cap
}  // namespace

dfamin_status device_props(int* dev_out, int* sms, size_t* smem_optin)
{
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return DFAMIN_ECUDA;
    if (dev_out) *dev_out = dev;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_props.find(dev);
    if (it == g_props.end()) {
        Props pr;
        int v = 0;
        if (!cuda_ok(cudaDeviceGetAttribute(&pr.sms, cudaDevAttrMultiProcessorCount, dev),
                     "cudaDeviceGetAttribute(SMs)"))
            return DFAMIN_ECUDA;
        if (!cuda_ok(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                     "cudaDeviceGetAttribute(smem)"))
            return DFAMIN_ECUDA;
        pr.smem_optin = (size_t)v;
        it = g_props.emplace(dev, pr).first;
    }
    if (sms) *sms = it->second.sms;
    if (smem_optin) *smem_optin = it->second.smem_optin;
    return DFAMIN_OK;
}

dfamin_status kernel_ctas_per_sm(int dev, const void* kernel, int threads, size_t smem, int* out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    // the kernel may use up to all the opt-in shared memory: set that once per device and
    // kernel (a smaller value set for one launch would refuse a later, larger one)
    const auto akey = std::make_pair(dev, kernel);
    if (!g_attr_set.count(akey)) {
        cudaFuncAttributes fa;
        if (!cuda_ok(cudaFuncGetAttributes(&fa, kernel), "cudaFuncGetAttributes")) return DFAMIN_ECUDA;
        int v = 0;
        if (!cuda_ok(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                     "cudaDeviceGetAttribute(smem)"))
            return DFAMIN_ECUDA;
        const int avail = v - (int)fa.sharedSizeBytes;
        if (!cuda_ok(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          avail > 0 ? avail : 0),
                     "cudaFuncSetAttribute(max dynamic shared memory)"))
            return DFAMIN_ECUDA;
        g_attr_set[akey] = avail;
    }
    if ((long long)smem > (long long)g_attr_set[akey]) return DFAMIN_EINVAL;
    const auto key = std::make_pair(akey, std::make_pair(threads, smem));
    auto it = g_occ.find(key);
    if (it != g_occ.end()) { *out = it->second; return DFAMIN_OK; }
    int b = 0;
    if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
        return DFAMIN_ECUDA;
    g_occ[key] = b;
    *out = b;
    return DFAMIN_OK;
}

}  // namespace dfamin_host

using namespace dfamin_host;
using namespace dfamin_dev;

namespace {

// Workspace of one DFA: [control | per-CTA counts | identity flags | DFA arrays | trace].
struct Layout {
    size_t ctrl, cta_cnt, nonid, pat, zero_end;  // [ctrl .. zero_end) is zeroed per launch
    size_t trace, dfa, total;
    DfaLayout d;
};

Layout make_layout(int32_t n, int32_t k, const dfamin_options& o)
{
    Layout L{};
    const size_t A = 256;
    size_t off = 0;
    L.ctrl = off; off = align_up(off + sizeof(Ctrl), A);
    L.cta_cnt = off; off = align_up(off + sizeof(int32_t) * kMaxCtas, A);
    L.nonid = off; off = align_up(off + sizeof(int32_t) * (size_t)(k > 0 ? k : 1), A);
    L.pat = off; off = align_up(off + sizeof(int32_t) * (size_t)kPatMax, A);
    L.zero_end = off;
    L.dfa = off;
    L.d = make_dfa_layout(n, k, o.closure == DFAMIN_CLOSURE_ON, true, o.closure_columns);
    off += L.d.total;
    L.trace = off;                          // the trace is the workspace's last bytes
    if (o.flags & DFAMIN_FLAG_TRACE) off += DFAMIN_TRACE_BYTES;
    L.total = off;
    return L;
}

// Alphabet sizes with a compile-time kernel; every other size, and every closure run, uses
// the runtime-width kernel team_kernel<0>.  *smem receives the kernel's dynamic shared memory.
template <int KC>
const void* team_entry(size_t* smem, int* threads)
{
    *smem = sizeof(typename CacheOf<KC>::type);
    *threads = TeamShape<KC>::threads;
    return (const void*)team_kernel<KC>;
}

const void* team_kernel_for(int k, bool closure, const int32_t* delta, size_t* smem, int* threads)
{
    const bool aligned = ((uintptr_t)delta & 15u) == 0;
    if (!closure && aligned) {
        switch (k) {
        case 1: return team_entry<1>(smem, threads);
        case 2: return team_entry<2>(smem, threads);
        case 3: return team_entry<3>(smem, threads);
        case 4: return team_entry<4>(smem, threads);
        case 5: return team_entry<5>(smem, threads);
        case 6: return team_entry<6>(smem, threads);
        case 7: return team_entry<7>(smem, threads);
        case 8: return team_entry<8>(smem, threads);
        default: break;
        }
    }
    *smem = 0;
    *threads = TeamShape<0>::threads;
    return (const void*)team_kernel<0>;
}

// Fills the device pointers of a DFA's arrays inside a workspace region.
void bind_dfa_arrays(Job& J, unsigned char* region, const DfaLayout& d)
{
    J.cl_letter = (int32_t*)(region + d.cl_letter);
    J.block = (int32_t*)(region + d.block);
    J.lst_s = (int32_t*)(region + d.lst_s);
    J.lst_slot = (uint32_t*)(region + d.lst_slot);
    J.lst_rst = (uint32_t*)(region + d.lst_rst);
    J.lead = (int32_t*)(region + d.lead);
    J.lead_slot = (uint32_t*)(region + d.lead_slot);
    J.stg = (int32_t*)(region + d.stg);
    J.naive_new = (int32_t*)(region + d.naive_new);
    J.spl = (int32_t*)(region + d.spl);
    J.cln = (int32_t*)(region + d.cln);
    J.table = (unsigned long long*)(region + d.table);
    J.mask = d.cap - 1;
    J.sig = (int32_t*)(region + d.sig);
    J.sig_stride = d.sig_stride;
    J.cl = (int32_t*)(region + d.cl);
    J.levels = d.levels;
    J.cl_cols = d.cols;
}

// End-to-end calls on host arrays: where the rows come from and where the labels go.  The
// aliases are the device-visible addresses of page-locked host memory, or null; what cannot be
// read or written in place by the kernel is copied in stream order around the launch.
struct HostIo {
    const int32_t* delta_h;         // host rows
    const int32_t* delta_alias;
    int32_t* out_h;                 // host labels
    int32_t* out_alias;
};

// The device-visible address of page-locked host memory (cudaHostAlloc, cudaHostRegister),
// or null for pageable memory.
void* host_alias(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// Stages what the chosen kernel does not move itself: rows before the launch (in = true), labels
// after it (in = false).
dfamin_status host_io_copy(const HostIo* io, bool in, bool kernel_moves_it, int32_t n, int32_t k,
                           int32_t* d_delta, int32_t* d_out, cudaStream_t stream)
{
    if (!io || kernel_moves_it) return DFAMIN_OK;
    if (in) {
        if (k > 0 && !cuda_ok(cudaMemcpyAsync(d_delta, io->delta_h,
                                              sizeof(int32_t) * (size_t)n * (size_t)k,
                                              cudaMemcpyHostToDevice, stream),
                              "cudaMemcpyAsync(rows to device)"))
            return DFAMIN_ECUDA;
        return DFAMIN_OK;
    }
    return cuda_ok(cudaMemcpyAsync(io->out_h, d_out, sizeof(int32_t) * (size_t)n,
                                   cudaMemcpyDeviceToHost, stream),
                   "cudaMemcpyAsync(labels to host)")
               ? DFAMIN_OK
               : DFAMIN_ECUDA;
}

dfamin_status launch_one(int32_t n, int32_t k, const int32_t* delta, const uint32_t* accept,
                         int32_t* out_block, int32_t* nblocks, const dfamin_options& o,
                         void* ws, size_t ws_bytes, int32_t* passes, int32_t* status,
                         cudaStream_t stream, const HostIo* io = nullptr)
{
    if (n < 1 || n > (1 << 30) || k < 0 || (int64_t)n * (int64_t)k >= ((int64_t)1 << 40))
        return DFAMIN_EINVAL;
    if ((k > 0 && !delta) || !accept || !out_block || !nblocks || !ws) return DFAMIN_EINVAL;
    if (((uintptr_t)ws & 255u) != 0 || ((uintptr_t)delta & 3u) != 0 ||
        ((uintptr_t)accept & 3u) != 0)
        return DFAMIN_EINVAL;
    dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    const Layout L = make_layout(n, k, o);
    if (ws_bytes < L.total) return DFAMIN_ENOMEM;
    int dev = 0, sms = 0;
    size_t smem_optin = 0;
    st = device_props(&dev, &sms, &smem_optin);
    if (st != DFAMIN_OK) return st;

    unsigned char* base = (unsigned char*)ws;
    Job J{};
    J.n = n;
    J.k = k;
    J.delta = delta;
    J.accept = accept;
    J.acc_off = 0;
    J.out_block = out_block;
    J.nblocks_out = nblocks;
    J.passes_out = passes;
    J.status_out = status;
    J.ctrl = (Ctrl*)(base + L.ctrl);
    J.cta_cnt = (int32_t*)(base + L.cta_cnt);
    J.nonid = (int32_t*)(base + L.nonid);
    J.pat_rev = (int32_t*)(base + L.pat);
    bind_dfa_arrays(J, base + L.dfa, L.d);
    J.max_passes = o.max_passes > 0 ? o.max_passes : (n < 0x7fffffff ? n + 1 : n);
    J.flags = o.flags;
    J.algo = o.algorithm;
    J.timeout_ns = o.barrier_timeout_us > 0 ? 1000ll * o.barrier_timeout_us : kBarrierTimeoutNs;
    if (o.flags & DFAMIN_FLAG_TRACE) {
        J.trace = (long long*)(base + L.trace);
        J.trace_cap = (DFAMIN_TRACE_BYTES / 8 - 1) / 2;
        if (!cuda_ok(cudaMemsetAsync(J.trace, 0, sizeof(long long), stream), "cudaMemsetAsync(trace)"))
            return DFAMIN_ECUDA;
    }

    if (!cuda_ok(cudaMemsetAsync(base + L.ctrl, 0, L.zero_end - L.ctrl, stream),
                 "cudaMemsetAsync(ctrl)"))
        return DFAMIN_ECUDA;

    const int small_limit = o.smem_states > 0 ? o.smem_states : 4096;
    uint32_t scap = 0;
    const size_t smem = small_smem_bytes(n, &scap);
    if (o.algorithm == DFAMIN_ALG_SIGNATURE && n <= small_limit && n <= kSmallMaxStates &&
        smem + 1024 <= smem_optin) {
        int per_sm = 0;
        st = kernel_ctas_per_sm(dev, (const void*)small_kernel, kThreads, smem, &per_sm);
        if (st != DFAMIN_OK) return st;
        st = host_io_copy(io, true, false, n, k, (int32_t*)delta, out_block, stream);
        if (st != DFAMIN_OK) return st;
        (void)cudaGetLastError();   // the check below must see this launch's error only
        small_kernel<<<1, kThreads, smem, stream>>>(J, scap);
        if (!cuda_ok(cudaGetLastError(), "small_kernel launch")) return DFAMIN_ECUDA;
        return host_io_copy(io, false, false, n, k, (int32_t*)delta, out_block, stream);
    }
    // one CTA with 16-bit ids and delta in shared memory (no closure): when asked
    // (smem_states >= n), or by default when a round's shared-memory work is small
    // (n * (2k + 1) <= 200,000), where it beats three grid barriers per round
    if (L.d.levels == 1 && n > (o.algorithm == DFAMIN_ALG_SIGNATURE ? kSmallMaxStates / 2 : 0) &&
        n <= kMediumMaxStates) {
        const bool pick = o.smem_states > 0 ? n <= o.smem_states
                                            : (int64_t)n * (2 * (int64_t)k + 1) <= 200000;
        const size_t msmem = align_up(sizeof(uint16_t) * (size_t)n * (size_t)(k + 1), 16);
        int per_sm = 0;
        if (pick && msmem + 1024 <= smem_optin &&
            kernel_ctas_per_sm(dev, (const void*)medium_kernel, kMediumThreads, msmem, &per_sm) ==
                DFAMIN_OK &&
            per_sm >= 1) {
            st = host_io_copy(io, true, false, n, k, (int32_t*)delta, out_block, stream);
            if (st != DFAMIN_OK) return st;
            (void)cudaGetLastError();
            medium_kernel<<<1, kMediumThreads, msmem, stream>>>(J);
            if (!cuda_ok(cudaGetLastError(), "medium_kernel launch")) return DFAMIN_ECUDA;
            return host_io_copy(io, false, false, n, k, (int32_t*)delta, out_block, stream);
        }
    }
    size_t dsmem = 0;
    int threads = 0;
    const void* kern = team_kernel_for(k, L.d.levels > 1, delta, &dsmem, &threads);
    int per_sm = 0;
    st = kernel_ctas_per_sm(dev, kern, threads, dsmem, &per_sm);
    if (st != DFAMIN_OK) return st;
    int max_ctas = sms * per_sm;
    if (max_ctas > kMaxCtas) max_ctas = kMaxCtas;
    if (max_ctas < 1) return DFAMIN_ECUDA;
    int ctas = o.ctas > 0 ? o.ctas : max_ctas;
    // at least ~2 states per thread per CTA: small DFAs use fewer CTAs (cheaper barriers)
    const int64_t want = ((int64_t)n + 2 * threads - 1) / (2 * threads);
    if (o.ctas == 0 && want < ctas) ctas = (int)(want > 0 ? want : 1);
    if (ctas > max_ctas) ctas = max_ctas;
    // end-to-end: round 1 of a compile-time alphabet reads every row itself (from host memory
    // when the rows are page-locked and aligned for its vector loads), and the canonical pass
    // writes the labels to page-locked host memory
    bool rows_in_kernel = false, labels_in_kernel = false;
    if (io) {
        const bool pattern_round = L.d.levels == 1 && o.algorithm == DFAMIN_ALG_SIGNATURE &&
                                   k >= 1 && k <= kPatMaxK;
        const uintptr_t need = (k % 4 == 0) ? 16 : ((k % 2 == 0) ? 8 : 4);
        rows_in_kernel = pattern_round && io->delta_alias &&
                         ((uintptr_t)io->delta_alias % need) == 0;
        labels_in_kernel = io->out_alias != nullptr;
        if (rows_in_kernel) {
            J.delta_host = io->delta_alias;
            J.delta_fill = (int32_t*)delta;
        }
        if (labels_in_kernel) J.out_host = io->out_alias;
    }
    st = host_io_copy(io, true, rows_in_kernel, n, k, (int32_t*)delta, out_block, stream);
    if (st != DFAMIN_OK) return st;
    void* args[] = {&J};
    if (!cuda_ok(cudaLaunchCooperativeKernel(kern, dim3(ctas), dim3(threads), args, dsmem,
                                             stream),
                 "team_kernel cooperative launch"))
        return DFAMIN_ECUDA;
    return host_io_copy(io, false, labels_in_kernel, n, k, (int32_t*)delta, out_block, stream);
}

// Workspace of an end-to-end call: device copies of the rows, the bitmap, the labels and the
// scalars, then the workspace of the minimization itself.
struct HostLayout {
    size_t delta, accept, out, sc, ws, total;
};

HostLayout host_layout(int32_t n, int32_t k, const dfamin_options& o)
{
    HostLayout H{};
    const size_t A = 256;
    size_t off = 0;
    H.delta = off; off = align_up(off + sizeof(int32_t) * (size_t)n * (size_t)k, A);
    H.accept = off; off = align_up(off + sizeof(uint32_t) * (((size_t)n + 31) / 32), A);
    H.out = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
    H.sc = off; off = align_up(off + 3 * sizeof(int32_t), A);
    H.ws = off;
    H.total = off + make_layout(n, k, o).total;
    return H;
}

// Scratch of dfamin_minimize_static: a file-scope device array (no allocation call).  Host code
// must not use its name as a device address; the address comes from cudaGetSymbolAddress,
// looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_static_scratch[DFAMIN_STATIC_SCRATCH_BYTES];
std::map<int, void*> g_static_addr;

dfamin_status static_scratch_address(void** out)
{
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return DFAMIN_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_static_addr.find(dev);
    if (it != g_static_addr.end()) { *out = it->second; return DFAMIN_OK; }
    void* ptr = nullptr;
    if (!cuda_ok(cudaGetSymbolAddress(&ptr, g_static_scratch), "cudaGetSymbolAddress(scratch)"))
        return DFAMIN_ECUDA;
    g_static_addr[dev] = ptr;
    *out = ptr;
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
    if (n < 1 || n > (1 << 30) || k < 0 || !bytes) return DFAMIN_EINVAL;
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
    if (n < 1 || n > (1 << 30) || k < 0) return DFAMIN_EINVAL;
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

DFAMIN_API dfamin_status dfamin_minimize_static(int32_t n, int32_t k, const int32_t* delta,
                                                const uint32_t* accept, int32_t* out_block,
                                                int32_t* nblocks, const dfamin_options* opt,
                                                int32_t* passes, int32_t* status,
                                                dfamin_stream_t stream)
{
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    if (n < 1 || n > (1 << 30) || k < 0) return DFAMIN_EINVAL;
    const dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    const size_t need = make_layout(n, k, o).total;
    if (need > (size_t)DFAMIN_STATIC_SCRATCH_BYTES) return DFAMIN_ENOMEM;
    void* scratch = nullptr;
    const dfamin_status sa = static_scratch_address(&scratch);
    if (sa != DFAMIN_OK) return sa;
    return launch_one(n, k, delta, accept, out_block, nblocks, o, scratch,
                      (size_t)DFAMIN_STATIC_SCRATCH_BYTES, passes, status, (cudaStream_t)stream);
}

DFAMIN_API dfamin_status dfamin_minimize_from_host_workspace_size(int32_t n, int32_t k,
                                                                   const dfamin_options* opt,
                                                                   size_t* bytes)
{
    if (n < 1 || n > (1 << 30) || k < 0 || !bytes) return DFAMIN_EINVAL;
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    const dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    *bytes = host_layout(n, k, o).total;
    return DFAMIN_OK;
}

DFAMIN_API dfamin_status dfamin_minimize_from_host(int32_t n, int32_t k, const int32_t* h_delta,
                                                   const uint32_t* h_accept, int32_t* h_out_block,
                                                   int32_t* h_scalars, const dfamin_options* opt,
                                                   void* workspace, size_t workspace_bytes,
                                                   dfamin_stream_t stream)
{
    if (n < 1 || n > (1 << 30) || k < 0) return DFAMIN_EINVAL;
    if ((k > 0 && !h_delta) || !h_accept || !h_out_block || !h_scalars || !workspace)
        return DFAMIN_EINVAL;
    if (((uintptr_t)workspace & 255u) != 0) return DFAMIN_EINVAL;
    dfamin_options o;
    dfamin_default_options(&o);
    if (opt) o = *opt;
    dfamin_status st = check_options(o);
    if (st != DFAMIN_OK) return st;
    const HostLayout H = host_layout(n, k, o);
    if (workspace_bytes < H.total) return DFAMIN_ENOMEM;
    unsigned char* base = (unsigned char*)workspace;
    int32_t* d_delta = (int32_t*)(base + H.delta);
    uint32_t* d_acc = (uint32_t*)(base + H.accept);
    int32_t* d_out = (int32_t*)(base + H.out);
    int32_t* d_sc = (int32_t*)(base + H.sc);
    // the bitmap first: round 1 looks up the acceptance of successors anywhere in it
    if (!cuda_ok(cudaMemcpyAsync(d_acc, h_accept, sizeof(uint32_t) * (((size_t)n + 31) / 32),
                                 cudaMemcpyHostToDevice, (cudaStream_t)stream),
                 "cudaMemcpyAsync(bitmap to device)"))
        return DFAMIN_ECUDA;
    HostIo io{h_delta, (const int32_t*)host_alias(h_delta), h_out_block,
              (int32_t*)host_alias(h_out_block)};
    int32_t* sc_alias = (int32_t*)host_alias(h_scalars);
    int32_t* sc = sc_alias ? sc_alias : d_sc;
    st = launch_one(n, k, d_delta, d_acc, d_out, sc, o, base + H.ws, workspace_bytes - H.ws,
                    sc + 1, sc + 2, (cudaStream_t)stream, &io);
    if (st != DFAMIN_OK) return st;
    if (!sc_alias && !cuda_ok(cudaMemcpyAsync(h_scalars, d_sc, 3 * sizeof(int32_t),
                                              cudaMemcpyDeviceToHost, (cudaStream_t)stream),
                              "cudaMemcpyAsync(scalars to host)"))
        return DFAMIN_ECUDA;
    return DFAMIN_OK;
}

DFAMIN_API const char* dfamin_last_cuda_error(void) { return dfamin_host::g_last_error; }

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

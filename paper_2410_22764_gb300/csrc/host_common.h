// Host-side helpers shared by the single-DFA entry points (dfamin.cu) and the batch entry
// points (batch.cu).  Include after refine.cuh (the layout uses its types).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

#include "dfamin.h"

#define DFAMIN_API extern "C" __attribute__((visibility("default")))

namespace dfamin_host {

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

inline dfamin_status check_options(const dfamin_options& o)
{
    if (o.closure != DFAMIN_CLOSURE_OFF && o.closure != DFAMIN_CLOSURE_ON) return DFAMIN_EINVAL;
    if (o.max_passes < 0 || o.ctas < 0 || o.smem_states < 0 || o.team_states < 0)
        return DFAMIN_EINVAL;
    if (o.algorithm != DFAMIN_ALG_SIGNATURE && o.algorithm != DFAMIN_ALG_LEADER)
        return DFAMIN_EINVAL;
    if (o.barrier_timeout_us < 0 || o.closure_columns < 0) return DFAMIN_EINVAL;
    return DFAMIN_OK;
}

// Shared memory of the one-CTA path: block ids, pending slots and the group table.
inline size_t small_smem_bytes(int32_t n, uint32_t* cap_out)
{
    const uint32_t cap = next_pow2_u32((uint64_t)n + (uint64_t)n / 2 + 32);
    if (cap_out) *cap_out = cap;
    return sizeof(int32_t) * 2 * (size_t)n + sizeof(uint32_t) * (size_t)cap;
}

// Per-DFA arrays of the multi-CTA path, as byte offsets from the start of the DFA's region.
struct DfaLayout {
    size_t block, lst_s, lst_slot, lst_rst, lead, lead_slot, stg, table, sig, cl, cl_letter,
        naive_new, spl, cln;
    size_t total;
    uint32_t cap;       // group-table capacity (power of two)
    int levels;         // 1 + floor(log2 n) with the closure, else 1
    int cols;           // closure columns held: k * (levels - 1), or the budget if smaller
    int sig_stride;     // ints per signature row
};

// col_budget: at most this many closure columns (0 = every column of every level).
inline DfaLayout make_dfa_layout(int32_t n, int32_t k, bool closure, bool arrays,
                                 int32_t col_budget = 0)
{
    DfaLayout L{};
    const size_t A = 256;
    size_t off = 0;
    L.levels = closure ? floor_log2(n) + 1 : 1;
    const int64_t full = (int64_t)k * (L.levels - 1);
    L.cols = (int)(col_budget > 0 && col_budget < full ? col_budget : full);
    const int64_t kmax = (int64_t)k + L.cols;        // signature columns (upper bound)
    L.sig_stride = (int)((kmax + 1 + 3) / 4 * 4);
    L.cap = next_pow2_u32((uint64_t)n + (uint64_t)n / 2 + 64);
    L.cl_letter = off; off = align_up(off + sizeof(int32_t) * (size_t)(k > 0 ? k : 1), A);
    if (arrays) {
        L.block = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.lst_s = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.lst_slot = off; off = align_up(off + sizeof(uint32_t) * (size_t)n, A);
        L.lst_rst = off; off = align_up(off + sizeof(uint32_t) * (size_t)n, A);
        L.lead = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.lead_slot = off; off = align_up(off + sizeof(uint32_t) * (size_t)n, A);
        L.stg = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.naive_new = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.spl = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.cln = off; off = align_up(off + sizeof(int32_t) * (size_t)n, A);
        L.table = off; off = align_up(off + sizeof(unsigned long long) * (size_t)L.cap, A);
        L.sig = off;
        off = align_up(off + sizeof(int32_t) * (size_t)n * (size_t)L.sig_stride, A);
    }
    L.cl = off;
    off = align_up(off + sizeof(int32_t) * (size_t)n * (size_t)L.cols, A);
    L.total = off;
    return L;
}

// Last CUDA failure seen by the calling thread (dfamin_last_cuda_error); false if e != success.
bool cuda_ok(cudaError_t e, const char* what);

extern std::mutex g_mu;

// Text of the calling thread's last failure (dfamin_last_cuda_error).
extern thread_local char g_last_error[256];

// Current device, its SM count and its per-block opt-in shared memory (cached per device).
dfamin_status device_props(int* dev, int* sms, size_t* smem_optin);

// CTAs of `kernel` that fit on one SM with `threads` threads and `smem` bytes of dynamic shared
// memory; sets the kernel's dynamic shared memory attribute on first use (cached per device).
dfamin_status kernel_ctas_per_sm(int dev, const void* kernel, int threads, size_t smem, int* out);

}  // namespace dfamin_host

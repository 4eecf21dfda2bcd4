// LTS -> DFA front end (arXiv 2410.22764, Sec. 4.1 "VLTSs"): a labelled transition system is
// made deterministic by the powerset construction from its initial state, then completed: every
// subset state accepts, and one extra non-accepting state (bottom) receives every transition
// the deterministic LTS lacks, and loops on every label.  The resulting DFA accepts the label
// sequences of the paths of the LTS from its initial state.
//
// Host code: it prepares inputs for the device minimizer and runs on the calling thread.
// Numbering: subset states get ids in the order a FIFO breadth-first search discovers them,
// taking labels in increasing order from each subset; {s0} is state 0; bottom is the last
// state.  This numbering is part of the contract (it makes the output reproducible).
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <unordered_map>
#include <utility>
#include <vector>

#include "dfamin.h"

#define DFAMIN_API extern "C" __attribute__((visibility("default")))

namespace {

struct SubsetHash {
    size_t operator()(const std::vector<int32_t>& v) const
    {
        // splitmix64 finalizer chained over the members (Steele, Lea & Flood 2014)
        uint64_t h = 0x9E3779B97F4A7C15ull ^ v.size();
        for (int32_t x : v) {
            uint64_t z = h + (uint64_t)(uint32_t)x + 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            h = z ^ (z >> 31);
        }
        return (size_t)h;
    }
};

}  // namespace

DFAMIN_API dfamin_status dfamin_lts_determinize(int32_t n, int32_t nlabels, int64_t m,
                                                const int32_t* src, const int32_t* lbl,
                                                const int32_t* dst, int32_t s0,
                                                int32_t max_states, int32_t* out_delta,
                                                uint32_t* out_accept, int32_t* out_n)
{
    if (!out_n) return DFAMIN_EINVAL;
    *out_n = 0;
    if (n < 1 || nlabels < 0 || m < 0 || s0 < 0 || s0 >= n || max_states < 1 ||
        (m > 0 && (!src || !lbl || !dst)) || !out_accept || (nlabels > 0 && !out_delta))
        return DFAMIN_EINVAL;
    if (max_states < 2) {                           // {s0} and bottom
        *out_n = -1;
        return DFAMIN_ENOMEM;
    }
    for (int64_t i = 0; i < m; ++i)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || lbl[i] < 0 ||
            lbl[i] >= nlabels)
            return DFAMIN_EINVAL;

    // transitions grouped by source, each group ordered by (label, target), duplicates removed
    std::vector<int64_t> row(n + 1, 0);
    for (int64_t i = 0; i < m; ++i) ++row[src[i] + 1];
    for (int32_t s = 0; s < n; ++s) row[s + 1] += row[s];
    std::vector<std::pair<int32_t, int32_t>> out((size_t)m);
    {
        std::vector<int64_t> fill(row.begin(), row.end() - 1);
        for (int64_t i = 0; i < m; ++i) out[(size_t)fill[src[i]]++] = {lbl[i], dst[i]};
    }
    for (int32_t s = 0; s < n; ++s)
        std::sort(out.begin() + row[s], out.begin() + row[s + 1]);

    std::unordered_map<std::vector<int32_t>, int32_t, SubsetHash> ids;
    std::vector<const std::vector<int32_t>*> subset;     // by id
    std::vector<int32_t> delta;                          // [ids][nlabels], -1 = bottom
    std::deque<int32_t> queue;
    {
        auto it = ids.emplace(std::vector<int32_t>{s0}, 0).first;
        subset.push_back(&it->first);
        queue.push_back(0);
    }
    std::vector<std::pair<int32_t, int32_t>> moves;
    std::vector<int32_t> target;
    while (!queue.empty()) {
        const int32_t id = queue.front();
        queue.pop_front();
        moves.clear();
        for (int32_t s : *subset[id])
            moves.insert(moves.end(), out.begin() + row[s], out.begin() + row[s + 1]);
        std::sort(moves.begin(), moves.end());
        moves.erase(std::unique(moves.begin(), moves.end()), moves.end());
        delta.resize((size_t)(id + 1) * (size_t)nlabels, -1);
        for (size_t i = 0; i < moves.size();) {
            const int32_t a = moves[i].first;
            target.clear();
            for (; i < moves.size() && moves[i].first == a; ++i) target.push_back(moves[i].second);
            auto found = ids.find(target);
            int32_t t;
            if (found != ids.end()) {
                t = found->second;
            } else {
                t = (int32_t)subset.size();
                if (t + 1 >= max_states) {          // no room for this state and bottom
                    *out_n = -1;
                    return DFAMIN_ENOMEM;
                }
                auto it = ids.emplace(target, t).first;
                subset.push_back(&it->first);
                queue.push_back(t);
            }
            delta[(size_t)id * (size_t)nlabels + (size_t)a] = t;
        }
    }
    const int32_t nsub = (int32_t)subset.size();
    const int32_t bottom = nsub;
    const int32_t total = nsub + 1;
    delta.resize((size_t)nsub * (size_t)nlabels, -1);
    for (size_t i = 0; i < delta.size(); ++i) out_delta[i] = delta[i] < 0 ? bottom : delta[i];
    for (int32_t a = 0; a < nlabels; ++a) out_delta[(size_t)bottom * nlabels + a] = bottom;
    memset(out_accept, 0, sizeof(uint32_t) * (size_t)((total + 31) / 32));
    for (int32_t q = 0; q < nsub; ++q) out_accept[q >> 5] |= 1u << (q & 31);
    *out_n = total;
    return DFAMIN_OK;
}

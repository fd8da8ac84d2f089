// registry.cpp -- flattening of the registered subnets into sorted disjoint ranges.
//
// The paper's Catalog Kernel expands every registered network into /24 entries of a
// hash table (Sec. III.B.2.1), which cannot express prefixes longer than /24 or a
// prefix nested inside another site's. Here the "Site Catalog" (Sec. III.B.1) becomes
// a partition of the whole IPv4 space into ranges [start_i, start_{i+1}), each carrying
// the site of the longest registered prefix that covers it (or no site). A lookup is
// then a predecessor search over the starts.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "gnm.h"
#include "hash24.hpp"

namespace gnm {

static inline uint32_t mask_of(unsigned len) { return len == 0 ? 0u : (0xFFFFFFFFu << (32u - len)); }

// Returns an empty string on success, else the reason the registry is invalid.
std::string flatten_registry(const uint32_t* prefix, const uint8_t* len, const uint32_t* site,
                             size_t n, uint32_t n_sites, std::vector<uint32_t>* starts,
                             std::vector<uint32_t>* sites) {
    struct P {
        uint32_t start;
        uint32_t len;
        uint32_t site;
        uint64_t end;
    };
    std::vector<P> v(n);
    for (size_t i = 0; i < n; ++i) {
        if (len[i] > 32) return "prefix " + std::to_string(i) + ": length > 32";
        if ((prefix[i] & ~mask_of(len[i])) != 0) return "prefix " + std::to_string(i) + ": host bits set";
        if (site[i] >= n_sites) return "prefix " + std::to_string(i) + ": site id >= n_sites";
        v[i] = P{prefix[i], len[i], site[i], (uint64_t)prefix[i] + (1ull << (32 - len[i]))};
    }
    // parents before children: by start, then shorter first
    std::sort(v.begin(), v.end(), [](const P& a, const P& b) {
        return a.start != b.start ? a.start < b.start : a.len < b.len;
    });
    for (size_t i = 1; i < n; ++i)
        if (v[i].start == v[i - 1].start && v[i].len == v[i - 1].len)
            return "duplicate prefix (same network and length)";

    starts->clear();
    sites->clear();
    auto emit = [&](uint64_t pos, uint32_t s) {
        if (pos >= (1ull << 32)) return;
        if (!starts->empty() && starts->back() == (uint32_t)pos) {
            sites->back() = s;  // a later boundary at the same address wins
            const size_t k = sites->size();
            if (k >= 2 && (*sites)[k - 2] == s) {
                starts->pop_back();
                sites->pop_back();
            }
            return;
        }
        if (!sites->empty() && sites->back() == s) return;  // merge equal neighbours
        starts->push_back((uint32_t)pos);
        sites->push_back(s);
    };
    emit(0, GNM_NO_SITE);
    std::vector<P> open;  // prefixes containing the sweep position, innermost last
    for (const P& p : v) {
        while (!open.empty() && open.back().end <= p.start) {
            const uint64_t e = open.back().end;
            open.pop_back();
            emit(e, open.empty() ? GNM_NO_SITE : open.back().site);
        }
        emit(p.start, p.site);
        open.push_back(p);
    }
    while (!open.empty()) {
        const uint64_t e = open.back().end;
        open.pop_back();
        emit(e, open.empty() ? GNM_NO_SITE : open.back().site);
    }
    return std::string();
}

// The paper's GPU Site Catalog (Sec. III.B.2.1): every registered network expanded into
// its /24 subnets, entered in a hash table keyed by the subnet (address >> 8). Shorter
// prefixes are entered first, so a nested longer prefix overwrites its parent's subnets and
// the table holds the longest match of every /24. Open addressing with linear probing over
// a power-of-two table at most half full; an entry is (subnet + 1, site), 0 = empty.
// Only registries whose prefixes are all /24 or shorter can be expanded (false otherwise).
bool build_hash24(const uint32_t* prefix, const uint8_t* len, const uint32_t* site, size_t n,
                  std::vector<uint32_t>* table, uint32_t* mask) {
    uint64_t subnets = 0;
    for (size_t i = 0; i < n; ++i) {
        if (len[i] > 24) return false;
        subnets += 1ull << (24u - len[i]);
    }
    uint64_t cap = 1024;
    while (cap < 2 * subnets) cap <<= 1;
    if (cap > (1ull << 26)) return false;  // beyond 2^25 subnets: more than the catalog's purpose
    table->assign(2 * cap, 0u);
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return len[a] < len[b]; });
    for (size_t i : order) {
        const uint32_t first = prefix[i] >> 8, count = 1u << (24u - len[i]);
        for (uint32_t k = first; k < first + count; ++k) {
            uint64_t h = hash24(k) & (cap - 1);
            while ((*table)[2 * h] != 0u && (*table)[2 * h] != k + 1u) h = (h + 1) & (cap - 1);
            (*table)[2 * h] = k + 1u;
            (*table)[2 * h + 1] = site[i];
        }
    }
    *mask = (uint32_t)(cap - 1);
    return true;
}

// True when the local prefix overlaps any registered prefix (one contains the other).
bool local_overlaps(uint32_t lp, uint8_t ll, const uint32_t* prefix, const uint8_t* len, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        const unsigned m = ll < len[i] ? ll : len[i];
        if ((lp & mask_of(m)) == (prefix[i] & mask_of(m))) return true;
    }
    return false;
}

}  // namespace gnm

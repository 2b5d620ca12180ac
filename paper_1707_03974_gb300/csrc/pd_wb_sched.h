// Host-side slot schedule of the warp-blocked spin-down table (plain C++, no
// CUDA): used by the table build in pd_basis.cu and compiled on its own by the
// CPU tests.
//
// Shared-memory bank groups.  A slot of the row pass is one shared load per
// lane, and costs as many wavefronts as the most used bank group among the
// lanes served together (distinct targets in one group conflict).  Two layouts:
//  * 16-byte elements (two staged fixed-point rows, or four float32 rows):
//    8 lanes (one quarter warp) at a time over 8 groups of 4 banks, group t % 8;
//  * 4-byte elements (one staged float32 row, for rows too long to stage two
//    fixed-point rows): all 32 lanes over the 32 banks, bank t % 32.
// The sums are exact integer sums (and float32 sums in a fixed order), so the
// order of a lane's hops within a segment is free.  Per lane set, the slots are
// filled in order: each slot takes a maximum matching of lanes to distinct
// groups (augmenting paths; lanes whose remaining hops fill every remaining
// slot first, groups with the most remaining hops preferred), and a lane that
// must place a hop but found no free group joins its least used group.  A local
// search then swaps two slots of one lane when that lowers the summed
// worst-group load of the two slots.  On the 4x4 half-filled table the 16-byte
// layout measures 5.3 wavefronts per gather (natural order 8.9, the local
// search alone 7.0).
#pragma once

#include <algorithm>
#include <cstdint>
#include <functional>
#include <vector>

namespace pd_wb {

struct BankLayout {
    int NL;  // lanes served together
    int G;   // bank groups
};

inline void match_slots(std::vector<int32_t> &grid, int slots, int l0, const BankLayout &bl) {
    const int NL = bl.NL, G = bl.G;
    auto at = [&](int l, int s) -> int32_t & { return grid[(size_t)l * slots + s]; };
    std::vector<std::vector<int32_t>> rem(NL);
    for (int i = 0; i < NL; ++i)
        for (int s = 0; s < slots; ++s)
            if (at(l0 + i, s) >= 0) rem[i].push_back(at(l0 + i, s));
    std::vector<int> dem(G), lanes(NL), gown(G), choice(NL), mult(G);
    for (int s = 0; s < slots; ++s) {
        const int R = slots - s;
        std::fill(dem.begin(), dem.end(), 0);
        for (int i = 0; i < NL; ++i)
            for (int32_t t : rem[i]) ++dem[t % G];
        for (int i = 0; i < NL; ++i) lanes[i] = i;
        std::stable_sort(lanes.begin(), lanes.end(), [&](int a, int b) {
            const bool ma = (int)rem[a].size() >= R, mb = (int)rem[b].size() >= R;
            if (ma != mb) return ma;
            return rem[a].size() > rem[b].size();
        });
        std::fill(gown.begin(), gown.end(), -1);
        std::fill(choice.begin(), choice.end(), -1);
        // augmenting path from lane i over groups not yet visited (seen)
        std::function<bool(int, uint32_t &)> augment = [&](int i, uint32_t &seen) -> bool {
            uint32_t have = 0;
            for (int32_t t : rem[i]) have |= 1u << (t % G);
            int opts[32], no = 0;
            for (int g = 0; g < G; ++g)
                if (have >> g & 1u) opts[no++] = g;
            std::stable_sort(opts, opts + no, [&](int a, int b) { return dem[a] > dem[b]; });
            for (int k = 0; k < no; ++k) {
                const int g = opts[k];
                if (seen >> g & 1u) continue;
                seen |= 1u << g;
                if (gown[g] < 0 || augment(gown[g], seen)) {
                    gown[g] = i;
                    choice[i] = g;
                    return true;
                }
            }
            return false;
        };
        for (int k = 0; k < NL; ++k) {
            uint32_t seen = 0;
            if (!rem[lanes[k]].empty()) augment(lanes[k], seen);
        }
        std::fill(mult.begin(), mult.end(), 0);
        for (int i = 0; i < NL; ++i)
            if (choice[i] >= 0) ++mult[choice[i]];
        for (int k = 0; k < NL; ++k) {
            const int i = lanes[k];
            if (choice[i] >= 0 || (int)rem[i].size() < R) continue;
            int best = -1;
            for (int32_t t : rem[i]) {
                const int g = t % G;
                if (best < 0 || mult[g] < mult[best] || (mult[g] == mult[best] && dem[g] > dem[best])) best = g;
            }
            choice[i] = best;
            ++mult[best];
        }
        for (int i = 0; i < NL; ++i) {
            at(l0 + i, s) = -1;
            if (choice[i] < 0) continue;
            for (size_t k = 0; k < rem[i].size(); ++k)
                if (rem[i][k] % G == choice[i]) {
                    at(l0 + i, s) = rem[i][k];
                    rem[i].erase(rem[i].begin() + (long)k);
                    break;
                }
        }
    }
}

inline void balance_banks(std::vector<int32_t> &grid, int slots, const BankLayout &bl) {
    if (slots < 2) return;
    const int NL = bl.NL, G = bl.G;
    for (int l0 = 0; l0 < 32; l0 += NL) {
        match_slots(grid, slots, l0, bl);
        std::vector<int> cnt((size_t)slots * G, 0);
        auto at = [&](int l, int s) -> int32_t & { return grid[(size_t)l * slots + s]; };
        for (int l = l0; l < l0 + NL; ++l)
            for (int s = 0; s < slots; ++s)
                if (at(l, s) >= 0) ++cnt[(size_t)s * G + at(l, s) % G];
        auto worst = [&](int s) {
            int m = 0;
            for (int g = 0; g < G; ++g) m = std::max(m, cnt[(size_t)s * G + g]);
            return m;
        };
        for (int pass = 0; pass < 4; ++pass) {
            bool improved = false;
            for (int l = l0; l < l0 + NL; ++l)
                for (int s1 = 0; s1 < slots; ++s1)
                    for (int s2 = s1 + 1; s2 < slots; ++s2) {
                        const int32_t a = at(l, s1), b = at(l, s2);
                        if (a == b) continue;
                        const int before = worst(s1) + worst(s2);
                        if (a >= 0) --cnt[(size_t)s1 * G + a % G], ++cnt[(size_t)s2 * G + a % G];
                        if (b >= 0) --cnt[(size_t)s2 * G + b % G], ++cnt[(size_t)s1 * G + b % G];
                        if (worst(s1) + worst(s2) < before) {
                            std::swap(at(l, s1), at(l, s2));
                            improved = true;
                        } else {
                            if (a >= 0) ++cnt[(size_t)s1 * G + a % G], --cnt[(size_t)s2 * G + a % G];
                            if (b >= 0) ++cnt[(size_t)s2 * G + b % G], --cnt[(size_t)s1 * G + b % G];
                        }
                    }
            if (!improved) break;
        }
    }
}

}  // namespace pd_wb

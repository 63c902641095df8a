// batched_plan.h -- host side of the batched Parlett-Higham path
// (batched.cu): the per-level task tables of a group of matrices with one
// leaf size.  Block anti-diagonal d of a matrix depends only on smaller
// anti-diagonals of the same matrix (Section 5.2), so each level d has one
// block-sum launch over the tiles (and K splits) of anti-diagonal d of every
// matrix with more than d blocks, then one leaf launch.  Host code only; the
// tests compile it on its own to check the tables and the workspace bound.
#pragma once

#include <algorithm>
#include <cstddef>
#include <vector>

namespace signtri {

// K splits per tile at most, and the CTAs a level's block-sum launch aims at
// (two resident CTAs per SM, two waves on 152 SMs).
constexpr int kBatchSplitMax = 32;
constexpr int kBatchTargetCtas = 4 * 152;

struct GemmTask {
    int m, I, J, kb0, kb1, slot;
};
struct LeafTask {
    int m, I, J, nsplit, slot0, pad;
};
struct DiagTask {
    int m, blk;
};

struct Plan {
    std::vector<DiagTask> diag;
    std::vector<GemmTask> gemm;
    std::vector<LeafTask> leaf;
    std::vector<int> gemm_off, leaf_off;   // per level d (size nbmax + 1)
    std::vector<int> poff, noff;           // per member: sign permutation and count offsets
    int nbmax = 0;
    size_t max_slots = 0;
    size_t perm_len = 0, npos_len = 0;
};

// members: indices (into the batch) of the matrices of this group
inline void make_plan(const std::vector<int> &ns, int B, Plan &p)
{
    const int cnt = (int)ns.size();
    std::vector<int> nb(cnt);
    p.nbmax = 0;
    p.poff.assign(cnt, 0);
    p.noff.assign(cnt, 0);
    for (int k = 0; k < cnt; k++) {
        nb[k] = (ns[k] + B - 1) / B;
        p.nbmax = std::max(p.nbmax, nb[k]);
        for (int b = 0; b < nb[k]; b++) p.diag.push_back({k, b});
        p.poff[k] = (int)p.perm_len;
        p.noff[k] = (int)p.npos_len;
        p.perm_len += (size_t)nb[k] * B;
        p.npos_len += (size_t)nb[k];
    }
    p.gemm_off.assign(p.nbmax + 1, 0);
    p.leaf_off.assign(p.nbmax + 1, 0);
    for (int d = 0; d <= p.nbmax; d++) {
        p.gemm_off[d] = (int)p.gemm.size();
        p.leaf_off[d] = (int)p.leaf.size();
        if (d < 1 || d >= p.nbmax) continue;
        long long tiles = 0;
        for (int k = 0; k < cnt; k++) tiles += std::max(0, nb[k] - d);
        const int kmax = d - 1;
        int ns = 0, kc = 1;
        if (kmax > 0 && tiles > 0) {
            ns = (int)std::max(1LL, std::min<long long>(kmax, (kBatchTargetCtas + tiles - 1) / tiles));
            ns = std::min(ns, kBatchSplitMax);
            kc = (kmax + ns - 1) / ns;
            ns = (kmax + kc - 1) / kc;
        }
        int slot = 0;
        for (int k = 0; k < cnt; k++)
            for (int I = 0; I + d < nb[k]; I++) {
                const int J = I + d;
                p.leaf.push_back({k, I, J, ns, slot, 0});
                for (int s = 0; s < ns; s++) {
                    const int kb0 = I + 1 + s * kc;
                    p.gemm.push_back({k, I, J, kb0, std::min(kb0 + kc, J), slot + s});
                }
                slot += ns;
            }
        p.max_slots = std::max(p.max_slots, (size_t)slot);
    }
    p.gemm_off[p.nbmax] = (int)p.gemm.size();
    p.leaf_off[p.nbmax] = (int)p.leaf.size();
}

inline size_t plan_bytes(const Plan &p, int B)
{
    return p.diag.size() * sizeof(DiagTask) + p.gemm.size() * sizeof(GemmTask) + p.leaf.size() * sizeof(LeafTask) +
           2 * std::max<size_t>(p.max_slots, 1) * B * B * sizeof(double) + p.perm_len * sizeof(short) +
           p.npos_len * sizeof(int) + 2 * p.poff.size() * sizeof(int) + 12 * 256;
}

// An upper bound of plan_bytes over every subset of the matrices ns (the
// call reserves workspace before the inertia scan decides which matrices run
// here).  A subset has fewer tiles per level, so make_plan may cut their K
// ranges finer, but at level d it makes at most tiles x min(d - 1,
// kBatchSplitMax) and at most kBatchTargetCtas + tiles partial slots (one block-sum
// task per slot), both growing with the tile count; the other tables only
// shrink with the subset.
inline size_t plan_bytes_bound(const std::vector<int> &ns, int B)
{
    std::vector<int> nb(ns.size());
    int nbmax = 0;
    size_t diag = 0, perm = 0, npos = 0;
    for (size_t k = 0; k < ns.size(); k++) {
        nb[k] = (ns[k] + B - 1) / B;
        nbmax = std::max(nbmax, nb[k]);
        diag += nb[k];
        perm += (size_t)nb[k] * B;
        npos += nb[k];
    }
    size_t leaf = 0, gemm = 0, slots = 0;
    for (int d = 1; d < nbmax; d++) {
        long long tiles = 0;
        for (size_t k = 0; k < ns.size(); k++) tiles += std::max(0, nb[k] - d);
        leaf += (size_t)tiles;
        const long long per = std::min(d - 1, kBatchSplitMax);
        const size_t lv = (size_t)std::min(tiles * per, (long long)kBatchTargetCtas + tiles);
        gemm += lv;
        slots = std::max(slots, lv);
    }
    return diag * sizeof(DiagTask) + gemm * sizeof(GemmTask) + leaf * sizeof(LeafTask) +
           2 * std::max<size_t>(slots, 1) * B * B * sizeof(double) + perm * sizeof(short) + npos * sizeof(int) +
           2 * ns.size() * sizeof(int) + 12 * 256;
}

}  // namespace signtri

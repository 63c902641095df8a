// gathered_layout.h -- host side of the needed residual of the mixed
// variants (mixed.cu): the gathered index order and the residual products'
// job lists, from the signs of the diagonal.  The needed entries of
// TU - UT (signs differ) and U^2 - I (signs agree) are products of strictly
// upper triangular factors, so a term t_ik u_kj (or u_ik u_kj, ...) vanishes
// unless i < k < j; the gathered order lets each job skip the K-blocks where
// every term vanishes.  Host code only; the tests compile it on its own to
// check the layout and the job lists.
#pragma once

#include <algorithm>
#include <utility>
#include <vector>

#include "tc_job.h"

namespace signtri {

struct GatheredLayout {
    int ng = 0;                  // gathered positions, padding included
    int rows_g = 0;              // ng plus the zero block
    std::vector<int> gmap;       // original index -> gathered position (n entries)
    std::vector<int> ginv;       // gathered position -> original index, -1 for padding (rows_g entries)
    std::vector<int> base;       // first gathered position of each superblock (superblocks + 1 entries)
    std::vector<TcJob> jobs;     // same-class jobs, then opposite-class jobs
    int n_same = 0, n_opp = 0;
    double kb_same = 0.0, kb_opp = 0.0;   // sum over jobs of used quadrants x K-blocks
};

// The gathered layout: per superblock of `super` indices the positives in
// order, padded to 64, then the negatives; the jobs pair two row blocks of
// one class and superblock with two column blocks of one class and
// superblock (a lone block pairs with the zero block at ng).  pos[i] != 0
// when t_ii > 0.
inline void build_gathered_layout(int n, const unsigned char *pos, int super, GatheredLayout &L)
{
    auto pad = [](int x) { return (x + 63) / 64 * 64; };
    const int nsb = (n + super - 1) / super;
    std::vector<int> gmap(n), base(nsb + 1, 0), cnt_pos(nsb, 0), cls_len[2];
    cls_len[0].assign(nsb, 0);
    cls_len[1].assign(nsb, 0);
    int g = 0;
    for (int sb = 0; sb < nsb; sb++) {
        const int i0 = sb * super, i1 = std::min(n, i0 + super);
        int np_ = 0;
        for (int i = i0; i < i1; i++) np_ += pos[i];
        const int A = pad(np_), Bn = pad(i1 - i0 - np_);
        base[sb] = g;
        cls_len[0][sb] = A;
        cls_len[1][sb] = Bn;
        int rp = 0, rn = 0;
        for (int i = i0; i < i1; i++) gmap[i] = pos[i] ? g + rp++ : g + A + rn++;
        g += A + Bn;
    }
    base[nsb] = g;
    L.ng = g;
    L.rows_g = g + 64;
    std::vector<int> ginv(L.rows_g, -1);
    for (int i = 0; i < n; i++) ginv[gmap[i]] = i;
    // block pairs per (superblock, class): row offsets, lone block with the zero block
    auto pairs_of = [&](int sb, int cls) {
        std::vector<std::pair<int, int>> v;
        const int start = base[sb] + (cls ? cls_len[0][sb] : 0), len = cls_len[cls][sb];
        for (int o = 0; o < len; o += 128) v.push_back({start + o, o + 64 < len ? start + o + 64 : L.ng});
        return v;
    };
    // original indices of each superblock's positives and negatives, ascending
    std::vector<std::vector<int>> porig(nsb), norig(nsb);
    for (int i = 0; i < n; i++) (pos[i] ? porig : norig)[i / super].push_back(i);
    // K range of a job: the products vanish unless row < k < column, so in the
    // rows' superblock the K-blocks before the first positive above the rows'
    // smallest index are skipped (positives come first there) and in the
    // columns' superblock those after the last negative below the columns'
    // largest index (negatives come last); what lies between stays (zeros)
    auto k_start = [&](int sr, int cr, int first) {
        if (cr == 0) return first / 64;
        const int rmin = ginv[first];
        const int cp = (int)(std::upper_bound(porig[sr].begin(), porig[sr].end(), rmin) - porig[sr].begin());
        return (base[sr] + cp) / 64;
    };
    auto k_end = [&](int sc, const std::pair<int, int> &cpair) {
        int last = -1;   // gathered position of the pair's last real column
        for (int gpos : {cpair.second, cpair.first})
            if (gpos < L.ng && last < 0)
                for (int q = gpos + 63; q >= gpos; q--)
                    if (ginv[q] >= 0) { last = q; break; }
        const int cmax = ginv[last];
        const int cn = (int)(std::lower_bound(norig[sc].begin(), norig[sc].end(), cmax) - norig[sc].begin());
        const int end = base[sc] + cls_len[0][sc] + cn;
        return (end + 63) / 64;
    };
    std::vector<TcJob> same, opp;
    double kb_same = 0.0, kb_opp = 0.0;
    // longest superblock spans first (load balance); one superblock pair's
    // jobs together (they share operand panels in L2)
    for (int span = nsb - 1; span >= 0; span--)
        for (int sr = 0; sr + span < nsb; sr++) {
            const int sc = sr + span;
            for (int cr = 0; cr < 2; cr++)
                for (int cc = 0; cc < 2; cc++) {
                    const auto rows = pairs_of(sr, cr), cols = pairs_of(sc, cc);
                    for (const auto &rp : rows)
                        for (const auto &cp : cols) {
                            TcJob j;
                            j.rt = rp.first; j.rb = rp.second; j.cl = cp.first; j.cr = cp.second;
                            j.kb0 = k_start(sr, cr, rp.first);
                            j.kb1 = std::max(j.kb0, k_end(sc, cp));
                            j.slot = 0; j.pad = 0;
                            const double used = (double)((rp.second < L.ng) + 1) * ((cp.second < L.ng) + 1);
                            if (cr == cc) { same.push_back(j); kb_same += used * (j.kb1 - j.kb0); }
                            else { opp.push_back(j); kb_opp += used * (j.kb1 - j.kb0); }
                        }
                }
        }
    L.n_same = (int)same.size();
    L.n_opp = (int)opp.size();
    L.kb_same = kb_same;
    L.kb_opp = kb_opp;
    same.insert(same.end(), opp.begin(), opp.end());
    L.jobs = std::move(same);
    L.gmap = std::move(gmap);
    L.ginv = std::move(ginv);
    L.base = std::move(base);
}

}  // namespace signtri

// reorder_schedule.h -- host side of the Parlett-Sylvester reorder by sign
// (ps_fp64.cu): which adjacent pairs (k, k+1) each round of Givens swaps
// exchanges (Section 2 reorders the Schur form so that the positive
// eigenvalues come first; Section 3 counts the swaps).  Host code only; the
// tests compile it on its own to check the schedule.
#pragma once

#include <vector_types.h>

#include <algorithm>
#include <utility>
#include <vector>

namespace signtri {

// Rounds of the stable partition by sign, by odd-even transposition: in
// round r every pair (k, k+1) with k = r mod 2 that holds a negative above a
// positive is swapped (the pairs of a round are disjoint).  Output: the flat
// list of the upper index k of each swapped pair, round by round, and the
// rounds' offsets into it (offsets[r] .. offsets[r+1]); a round may be
// empty, and trailing empty rounds are dropped.  The number of swaps is
// #{i<j : t_ii < 0 < t_jj}, the minimum.
inline void schedule_rounds(const std::vector<double> &diag, std::vector<int> &pairs, std::vector<int> &offsets)
{
    const int n = (int)diag.size();
    std::vector<signed char> s(n);
    for (int i = 0; i < n; i++) s[i] = diag[i] > 0.0 ? 1 : -1;
    pairs.clear();
    offsets.assign(1, 0);
    int lo = 0, hi = n - 1;                       // unsorted window
    int idle = 0;
    for (int r = 0; idle < 2; r++) {
        while (lo < n && s[lo] > 0) lo++;         // leading positives are final
        while (hi >= 0 && s[hi] < 0) hi--;        // trailing negatives are final
        bool any = false;
        const int start = std::max(0, lo - 1);
        for (int k = start + ((start & 1) != (r & 1) ? 1 : 0); k + 1 <= hi; k += 2) {
            if (s[k] < 0 && s[k + 1] > 0) {
                std::swap(s[k], s[k + 1]);
                pairs.push_back(k);
                any = true;
            }
        }
        offsets.push_back((int)pairs.size());
        idle = any ? 0 : idle + 1;
    }
    while (offsets.size() > 1 && offsets[offsets.size() - 1] == offsets[offsets.size() - 2]) offsets.pop_back();
}

// Windowed form of the same stable partition (blocked reorder): sweeps over
// windows of w consecutive indices (w a multiple of 64, at most 128), their
// boundaries at offset 0 in even sweeps and w / 2 in odd ones (a first window
// of w / 2 then); in a sweep every window holding a negative above a positive
// is stable-partitioned on its own (positives first), by adjacent swaps.
// Output: per sweep the active windows (start, width); the total swap count
// (the same minimum k).  Ends when the whole sequence is partitioned.
inline void schedule_window_sweeps(const std::vector<double> &diag, int w, std::vector<std::vector<int2>> &sweeps,
                                   long long &swaps)
{
    const int n = (int)diag.size();
    std::vector<signed char> s(n);
    for (int i = 0; i < n; i++) s[i] = diag[i] > 0.0 ? 1 : -1;
    sweeps.clear();
    swaps = 0;
    auto sorted = [&]() {
        int i = 0;
        while (i < n && s[i] > 0) i++;
        while (i < n && s[i] < 0) i++;
        return i == n;
    };
    for (int t = 0; !sorted(); t++) {
        const int off = (t & 1) ? w / 2 : 0;
        std::vector<int2> act;
        for (int a = 0; a < n;) {
            const int b = std::min(n, a == 0 && off > 0 ? off : a + w);
            // inversions inside [a, b): pairs (negative, later positive)
            long long inv = 0, neg = 0;
            for (int i = a; i < b; i++) {
                if (s[i] < 0) neg++;
                else inv += neg;
            }
            if (inv > 0) {
                act.push_back(int2{a, b - a});
                swaps += inv;
                std::stable_partition(s.begin() + a, s.begin() + b, [](signed char x) { return x > 0; });
            }
            a = b;
        }
        sweeps.push_back(act);
    }
}

}  // namespace signtri

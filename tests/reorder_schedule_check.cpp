// Invariants of the Parlett-Sylvester reorder schedule (reorder_schedule.h)
// for seeded sign patterns of many sizes, by replaying the swaps on the
// signs and on the original indices:
//   - every swap exchanges a negative at k with a positive at k+1 (so each
//     one is a swap the reorder needs, Section 2);
//   - within a round the pairs are disjoint, ascending and of the round's
//     parity (k = r mod 2: the rotation kernels tell a pair's first index
//     from the round's parity);
//   - after the last round the positives come first, each sign group in its
//     original order (a stable partition);
//   - the number of swaps is #{i<j : s_i < 0 < s_j} (Section 3, the minimum);
//   - at most n + 1 rounds, offsets consistent, no trailing empty round;
// and of the windowed form (blocked reorder), by replaying its sweeps:
//   - windows disjoint, ascending, inside [0, n), starting on multiples of
//     w / 2 (the 64-row panels of the products that apply them), at most w
//     wide, each holding an inversion when its sweep comes;
//   - after the last sweep the same stable partition, with the same total
//     swap count; at most 2 n / (w / 2) + 2 sweeps.
// Prints "ok <swaps checked>" and exits 0, or the first violations and exit
// code 1.  Test infrastructure: compiled and run by the CPU tests.
#include <cstdio>
#include <random>
#include <vector>

#include "reorder_schedule.h"

using namespace signtri;

static int g_n = 0, g_case = 0, g_fails = 0;
static long long g_swaps = 0;

#define CHECK(cond, ...)                                                    \
    do {                                                                    \
        if (!(cond)) {                                                      \
            if (g_fails++ < 20) {                                           \
                std::printf("FAIL n=%d case %d line %d: ", g_n, g_case, __LINE__); \
                std::printf(__VA_ARGS__);                                   \
                std::printf("\n");                                          \
            }                                                               \
        }                                                                   \
    } while (0)

static void check(const std::vector<int> &sign)
{
    const int n = (int)sign.size();
    std::vector<double> diag(n);
    for (int i = 0; i < n; i++) diag[i] = sign[i] > 0 ? 0.5 + i % 7 : -0.5 - i % 5;
    std::vector<int> pairs, offsets;
    schedule_rounds(diag, pairs, offsets);
    long long inversions = 0, neg_seen = 0;
    for (int i = 0; i < n; i++) {
        if (sign[i] < 0) neg_seen++;
        else inversions += neg_seen;
    }
    CHECK((long long)pairs.size() == inversions, "%zu swaps, %lld inversions", pairs.size(), inversions);
    CHECK(!offsets.empty() && offsets[0] == 0 && offsets.back() == (int)pairs.size(), "offsets do not span the pairs");
    const int rounds = (int)offsets.size() - 1;
    CHECK(rounds <= n + 1, "%d rounds", rounds);
    CHECK(rounds == 0 || offsets[rounds] > offsets[rounds - 1], "trailing empty round");
    if (g_fails) return;
    std::vector<int> s = sign, orig(n);
    for (int i = 0; i < n; i++) orig[i] = i;
    for (int r = 0; r < rounds; r++) {
        CHECK(offsets[r] <= offsets[r + 1], "round %d: offsets decrease", r);
        int prev = -2;
        for (int q = offsets[r]; q < offsets[r + 1]; q++) {
            const int k = pairs[q];
            g_swaps++;
            CHECK(k >= 0 && k + 1 < n, "round %d: pair %d", r, k);
            if (k < 0 || k + 1 >= n) return;
            CHECK((k & 1) == (r & 1), "round %d: pair %d of the other parity", r, k);
            CHECK(k >= prev + 2, "round %d: pair %d overlaps pair %d", r, k, prev);
            CHECK(s[k] < 0 && s[k + 1] > 0, "round %d: pair %d holds signs %d, %d", r, k, s[k], s[k + 1]);
            std::swap(s[k], s[k + 1]);
            std::swap(orig[k], orig[k + 1]);
            prev = k;
        }
    }
    int npos = 0;
    for (int i = 0; i < n; i++) npos += sign[i] > 0;
    for (int i = 0; i < n; i++) CHECK((s[i] > 0) == (i < npos), "position %d holds sign %d after the rounds", i, s[i]);
    for (int i = 0; i + 1 < n; i++)
        if ((i + 1 < npos) || (i >= npos)) CHECK(orig[i] < orig[i + 1], "positions %d, %d out of original order", i, i + 1);

    // windowed sweeps
    constexpr int w = 128;
    std::vector<std::vector<int2>> sweeps;
    long long wswaps = 0;
    schedule_window_sweeps(diag, w, sweeps, wswaps);
    CHECK(wswaps == inversions, "windowed: %lld swaps, %lld inversions", wswaps, inversions);
    CHECK((long long)sweeps.size() <= 2LL * n / (w / 2) + 2, "windowed: %zu sweeps", sweeps.size());
    std::vector<int> ws = sign, worig(n);
    for (int i = 0; i < n; i++) worig[i] = i;
    for (size_t t = 0; t < sweeps.size(); t++) {
        int end = 0;
        for (const int2 &win : sweeps[t]) {
            const int a = win.x, b = win.x + win.y;
            CHECK(a >= end && win.y > 0 && win.y <= w && b <= n, "sweep %zu: window (%d, %d)", t, a, win.y);
            CHECK(a % (w / 2) == 0, "sweep %zu: window start %d", t, a);
            if (a < end || a < 0 || b > n || win.y <= 0) return;
            end = b;
            long long inv = 0, neg = 0;
            for (int i = a; i < b; i++) {
                if (ws[i] < 0) neg++;
                else inv += neg;
            }
            CHECK(inv > 0, "sweep %zu: window (%d, %d) already partitioned", t, a, win.y);
            std::vector<int> pos_s, neg_s, pos_o, neg_o;
            for (int i = a; i < b; i++) {
                (ws[i] > 0 ? pos_s : neg_s).push_back(ws[i]);
                (ws[i] > 0 ? pos_o : neg_o).push_back(worig[i]);
            }
            int i = a;
            for (size_t q = 0; q < pos_s.size(); q++, i++) { ws[i] = pos_s[q]; worig[i] = pos_o[q]; }
            for (size_t q = 0; q < neg_s.size(); q++, i++) { ws[i] = neg_s[q]; worig[i] = neg_o[q]; }
        }
    }
    for (int i = 0; i < n; i++) CHECK((ws[i] > 0) == (i < npos), "windowed: position %d holds sign %d", i, ws[i]);
    for (int i = 0; i + 1 < n; i++)
        if ((i + 1 < npos) || (i >= npos))
            CHECK(worig[i] < worig[i + 1], "windowed: positions %d, %d out of original order", i, i + 1);
}

int main()
{
    std::mt19937 rng(7);
    for (int n = 0; n <= 130; n++) {
        g_n = n;
        for (int c = 0; c < 12; c++) {
            g_case = c;
            std::vector<int> s(n);
            const double p = c / 11.0;
            for (int i = 0; i < n; i++) s[i] = std::uniform_real_distribution<double>(0, 1)(rng) < p ? -1 : 1;
            check(s);
        }
    }
    for (int n : {257, 1000, 1023, 2048, 3001}) {
        g_n = n;
        for (int c = 0; c < 8; c++) {
            g_case = c;
            std::vector<int> s(n);
            for (int i = 0; i < n; i++) {
                switch (c) {
                case 0: s[i] = i & 1 ? 1 : -1; break;                        // alternating, negative first
                case 1: s[i] = i < n / 2 ? -1 : 1; break;                    // all negatives above all positives
                case 2: s[i] = i < n / 2 ? 1 : -1; break;                    // already partitioned
                case 3: s[i] = -1; break;
                case 4: s[i] = 1; break;
                default: s[i] = std::uniform_real_distribution<double>(0, 1)(rng) < 0.1 * c ? -1 : 1;
                }
            }
            check(s);
        }
    }
    if (g_fails) {
        std::printf("%d violations\n", g_fails);
        return 1;
    }
    std::printf("ok %lld\n", g_swaps);
    return 0;
}

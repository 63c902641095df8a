// Invariants of the batched Parlett-Higham task tables (batched_plan.h) for
// seeded batches of uneven sizes and every leaf size:
//   - one diagonal-leaf task per diagonal block of every matrix;
//   - at level d one leaf task per tile (I, I+d) of every matrix with more
//     than d blocks, and block-sum tasks that cover the K-blocks strictly
//     between I and I+d (Section 5.2) exactly once, each in its own partial
//     slot inside the tile's slot range, the ranges disjoint and below
//     max_slots; the level offsets delimit exactly the level's tasks;
//   - the sign-permutation and count offsets are the prefix sums of the
//     matrices' padded sizes;
//   - plan_bytes_bound(ns) is at least plan_bytes of the plan of every subset
//     of ns (the batched call reserves workspace before it knows which of its
//     matrices run this path).
// Prints "ok <tasks checked>" and exits 0, or the first violations and exit
// code 1.  Test infrastructure: compiled and run by the CPU tests.
#include <cstdio>
#include <random>
#include <vector>

#include "batched_plan.h"

using namespace signtri;

static int g_case = 0, g_fails = 0;
static long long g_tasks = 0;

#define CHECK(cond, ...)                                              \
    do {                                                              \
        if (!(cond)) {                                                \
            if (g_fails++ < 20) {                                     \
                std::printf("FAIL case %d line %d: ", g_case, __LINE__); \
                std::printf(__VA_ARGS__);                             \
                std::printf("\n");                                    \
            }                                                         \
        }                                                             \
    } while (0)

static void check_plan(const std::vector<int> &ns, int B)
{
    Plan p;
    make_plan(ns, B, p);
    const int cnt = (int)ns.size();
    std::vector<int> nb(cnt);
    int nbmax = 0;
    size_t perm = 0, npos = 0;
    for (int k = 0; k < cnt; k++) {
        nb[k] = (ns[k] + B - 1) / B;
        nbmax = std::max(nbmax, nb[k]);
        CHECK(p.poff[k] == (int)perm && p.noff[k] == (int)npos, "matrix %d: offsets %d %d", k, p.poff[k], p.noff[k]);
        perm += (size_t)nb[k] * B;
        npos += nb[k];
    }
    CHECK(p.nbmax == nbmax && p.perm_len == perm && p.npos_len == npos, "sizes");
    // diagonal leaves
    std::vector<std::vector<int>> dseen(cnt);
    for (int k = 0; k < cnt; k++) dseen[k].assign(nb[k], 0);
    for (const DiagTask &t : p.diag) {
        CHECK(t.m >= 0 && t.m < cnt && t.blk >= 0 && t.blk < nb[t.m], "diagonal task (%d, %d)", t.m, t.blk);
        if (t.m >= 0 && t.m < cnt && t.blk >= 0 && t.blk < nb[t.m]) dseen[t.m][t.blk]++;
    }
    for (int k = 0; k < cnt; k++)
        for (int b = 0; b < nb[k]; b++) CHECK(dseen[k][b] == 1, "matrix %d block %d: %d diagonal tasks", k, b, dseen[k][b]);
    CHECK((int)p.gemm_off.size() == nbmax + 1 && (int)p.leaf_off.size() == nbmax + 1, "level offsets");
    if (g_fails) return;
    CHECK(p.gemm_off[0] == 0 && p.leaf_off[0] == 0, "level offsets start");
    for (int d = 0; d < nbmax; d++)
        CHECK(p.gemm_off[d] <= p.gemm_off[d + 1] && p.leaf_off[d] <= p.leaf_off[d + 1], "level %d offsets", d);
    CHECK(p.gemm_off[nbmax] == (int)p.gemm.size() && p.leaf_off[nbmax] == (int)p.leaf.size(), "level offsets end");
    CHECK(p.leaf_off[1] == 0 && p.gemm_off[1] == 0, "tasks at level 0");
    if (g_fails) return;
    for (int d = 1; d < nbmax; d++) {
        // the level's tiles: (matrix, I) -> leaf task
        std::vector<std::vector<int>> leaf_of(cnt);
        for (int k = 0; k < cnt; k++) leaf_of[k].assign(std::max(0, nb[k] - d), -1);
        std::vector<int> slot_used(std::max<size_t>(p.max_slots, 1), 0);
        for (int q = p.leaf_off[d]; q < p.leaf_off[d + 1]; q++) {
            const LeafTask &t = p.leaf[q];
            g_tasks++;
            CHECK(t.m >= 0 && t.m < cnt && t.J == t.I + d && t.I >= 0 && t.J < nb[t.m], "level %d leaf (%d, %d, %d)",
                  d, t.m, t.I, t.J);
            if (!(t.m >= 0 && t.m < cnt && t.I >= 0 && t.I + d < nb[t.m])) return;
            CHECK(leaf_of[t.m][t.I] < 0, "level %d: tile (%d, %d) of matrix %d twice", d, t.I, t.J, t.m);
            leaf_of[t.m][t.I] = q;
            CHECK(t.nsplit >= 0 && t.nsplit <= kBatchSplitMax && t.slot0 >= 0 &&
                      (size_t)(t.slot0 + t.nsplit) <= p.max_slots,
                  "level %d: slots [%d, +%d) of %zu", d, t.slot0, t.nsplit, p.max_slots);
            CHECK((d == 1) == (t.nsplit == 0), "level %d: %d splits", d, t.nsplit);
            for (int s = t.slot0; s < t.slot0 + t.nsplit && s < (int)slot_used.size(); s++) {
                CHECK(slot_used[s] == 0, "level %d: slot %d in two tiles", d, s);
                slot_used[s] = 1;
            }
        }
        for (int k = 0; k < cnt; k++)
            for (int I = 0; I + d < nb[k]; I++) CHECK(leaf_of[k][I] >= 0, "level %d: tile (%d, %d) of matrix %d missing", d, I, I + d, k);
        if (g_fails) return;
        // block sums: K-blocks strictly between, once each, in the tile's slots
        std::vector<std::vector<std::vector<int>>> kcov(cnt);
        for (int k = 0; k < cnt; k++) kcov[k].assign(std::max(0, nb[k] - d), std::vector<int>(d + 1, 0));
        std::vector<int> slot_task(slot_used.size(), 0);
        for (int q = p.gemm_off[d]; q < p.gemm_off[d + 1]; q++) {
            const GemmTask &g = p.gemm[q];
            g_tasks++;
            CHECK(g.m >= 0 && g.m < cnt && g.J == g.I + d && g.I >= 0 && g.J < nb[g.m], "level %d block sum (%d, %d, %d)",
                  d, g.m, g.I, g.J);
            if (!(g.m >= 0 && g.m < cnt && g.I >= 0 && g.I + d < nb[g.m])) return;
            CHECK(g.kb0 > g.I && g.kb0 < g.kb1 && g.kb1 <= g.J, "level %d: K [%d, %d) for tile (%d, %d)", d, g.kb0, g.kb1,
                  g.I, g.J);
            for (int kb = std::max(g.kb0, g.I); kb < g.kb1 && kb <= g.J; kb++) kcov[g.m][g.I][kb - g.I]++;
            const LeafTask &t = p.leaf[leaf_of[g.m][g.I]];
            CHECK(g.slot >= t.slot0 && g.slot < t.slot0 + t.nsplit, "level %d: slot %d outside [%d, +%d)", d, g.slot,
                  t.slot0, t.nsplit);
            if (g.slot >= 0 && g.slot < (int)slot_task.size()) {
                CHECK(slot_task[g.slot] == 0, "level %d: slot %d written twice", d, g.slot);
                slot_task[g.slot] = 1;
            }
        }
        for (int k = 0; k < cnt; k++)
            for (int I = 0; I + d < nb[k]; I++)
                for (int o = 0; o <= d; o++) {
                    const int want = (o > 0 && o < d) ? 1 : 0;
                    CHECK(kcov[k][I][o] == want, "level %d matrix %d tile %d: K-block +%d summed %d times", d, k, I, o,
                          kcov[k][I][o]);
                }
    }
}

int main()
{
    std::mt19937 rng(11);
    for (int c = 0; c < 400; c++) {
        g_case = c;
        const int B = 16 << (c % 3);
        const int cnt = 1 + (int)(rng() % (c < 300 ? 12 : 60));
        std::vector<int> ns(cnt);
        for (auto &x : ns) x = 1 + (int)(rng() % (c < 300 ? 700 : 2048));
        check_plan(ns, B);
        // the workspace bound against subsets
        const size_t bound = plan_bytes_bound(ns, B);
        for (int t = 0; t < 30; t++) {
            std::vector<int> sub;
            for (int x : ns)
                if (t == 0 || rng() % 3) sub.push_back(x);
            if (sub.empty()) continue;
            Plan p;
            make_plan(sub, B, p);
            CHECK(plan_bytes(p, B) <= bound, "subset of %zu of %d matrices needs %zu > bound %zu", sub.size(), cnt,
                  plan_bytes(p, B), bound);
        }
    }
    if (g_fails) {
        std::printf("%d violations\n", g_fails);
        return 1;
    }
    std::printf("ok %lld\n", g_tasks);
    return 0;
}

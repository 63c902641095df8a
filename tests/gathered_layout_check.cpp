// Invariants of the needed residual's gathered layout and job lists
// (gathered_layout.h), for seeded sign patterns of many sizes:
//   - the gathered order: per superblock the positives in original order,
//     padded to 64, then the negatives in order, padded to 64; gmap and ginv
//     inverse to each other, -1 on padding and on the zero block;
//   - every pair of 64-blocks (rows R, columns C) with R's superblock not
//     after C's lies in exactly one job, the others in none (so every needed
//     entry (i, j), i < j, is produced once); a job's two row blocks (and two
//     column blocks) are consecutive blocks of one superblock and class, a
//     lone block paired with the zero block;
//   - the K trimming drops no term: a product of strictly upper triangular
//     factors has terms only for row < k < column (original indices), and
//     every real k outside a job's K range has k <= the job's smallest row
//     or k >= its largest column;
//   - same-class jobs first, the quadrant x K-block sums match the jobs, and
//     the sizes fit the workspace the library reserves.
// Prints "ok <terms checked>" and exits 0, or the first violations and exit
// code 1.  Test infrastructure: compiled and run by the CPU tests.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "gathered_layout.h"

using namespace signtri;

constexpr int kSuperblock = 1024;   // the library's superblock of the gathered order

static int g_n = 0, g_case = 0, g_fails = 0;
static long long g_checked = 0;

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

static int pad64(int x) { return (x + 63) / 64 * 64; }

static void check(int n, const std::vector<unsigned char> &pos)
{
    GatheredLayout L;
    build_gathered_layout(n, pos.data(), kSuperblock, L);
    const int nsb = (n + kSuperblock - 1) / kSuperblock;
    // sizes against the workspace (gathered_bound and the job list bound)
    const long long gbound = pad64(n) + 128LL * nsb, ngr = gbound + 64;
    const long long pairs_max = ngr / 128 + 2LL * nsb + 2;
    CHECK(L.rows_g == L.ng + 64 && L.rows_g <= gbound + 64, "rows_g %d, ng %d, bound %lld", L.rows_g, L.ng, gbound);
    CHECK((long long)L.jobs.size() <= pairs_max * pairs_max, "%zu jobs, room for %lld", L.jobs.size(),
          pairs_max * pairs_max);
    CHECK((int)L.gmap.size() == n && (int)L.ginv.size() == L.rows_g && (int)L.base.size() == nsb + 1,
          "table sizes %zu %zu %zu", L.gmap.size(), L.ginv.size(), L.base.size());
    CHECK(L.n_same + L.n_opp == (int)L.jobs.size(), "%d + %d jobs of %zu", L.n_same, L.n_opp, L.jobs.size());
    if (g_fails) return;
    // the gathered order
    std::vector<int> expect(L.rows_g, -1);
    int g = 0;
    for (int sb = 0; sb < nsb; sb++) {
        CHECK(L.base[sb] == g, "superblock %d starts at %d, expected %d", sb, L.base[sb], g);
        const int i0 = sb * kSuperblock, i1 = std::min(n, i0 + kSuperblock);
        int q = g;
        for (int i = i0; i < i1; i++)
            if (pos[i]) expect[q++] = i;
        q = g + pad64(q - g);
        const int neg0 = q;
        for (int i = i0; i < i1; i++)
            if (!pos[i]) expect[q++] = i;
        g = neg0 + pad64(q - neg0);
    }
    CHECK(L.base[nsb] == g && L.ng == g, "end %d, ng %d, expected %d", L.base[nsb], L.ng, g);
    for (int q = 0; q < L.rows_g && q < (int)expect.size(); q++)
        CHECK(L.ginv[q] == expect[q], "ginv[%d] = %d, expected %d", q, L.ginv[q], expect[q]);
    for (int i = 0; i < n; i++) CHECK(L.gmap[i] >= 0 && L.gmap[i] < L.ng && L.ginv[L.gmap[i]] == i, "gmap[%d]", i);
    if (g_fails) return;
    // block coverage and job shapes
    const int nblk = L.ng / 64;
    auto sb_of = [&](int blk) {   // superblock of a gathered block
        int sb = 0;
        while (sb + 1 < nsb && L.base[sb + 1] <= blk * 64) sb++;
        return sb;
    };
    auto class_of = [&](int blk) {  // 0: positives, 1: negatives (from a real entry of the block)
        for (int q = blk * 64; q < blk * 64 + 64; q++)
            if (L.ginv[q] >= 0) return pos[L.ginv[q]] ? 0 : 1;
        return -1;
    };
    std::vector<int> bsb(nblk), bcls(nblk);
    for (int b = 0; b < nblk; b++) {
        bsb[b] = sb_of(b);
        bcls[b] = class_of(b);
        CHECK(bcls[b] >= 0, "gathered block %d holds no index", b);
    }
    std::vector<int> cover((size_t)nblk * nblk, 0);
    double kb_same = 0.0, kb_opp = 0.0;
    for (size_t jx = 0; jx < L.jobs.size(); jx++) {
        const TcJob &j = L.jobs[jx];
        int rows[2] = {j.rt / 64, j.rb < L.ng ? j.rb / 64 : -1};
        int cols[2] = {j.cl / 64, j.cr < L.ng ? j.cr / 64 : -1};
        CHECK(j.rt % 64 == 0 && j.cl % 64 == 0 && j.rb % 64 == 0 && j.cr % 64 == 0, "job %zu not block aligned", jx);
        CHECK(j.rt < L.ng && j.cl < L.ng && j.rb <= L.ng && j.cr <= L.ng, "job %zu outside the layout", jx);
        if (g_fails) return;
        CHECK(rows[1] < 0 || (rows[1] == rows[0] + 1 && bsb[rows[1]] == bsb[rows[0]] && bcls[rows[1]] == bcls[rows[0]]),
              "job %zu: row blocks %d, %d", jx, rows[0], rows[1]);
        CHECK(cols[1] < 0 || (cols[1] == cols[0] + 1 && bsb[cols[1]] == bsb[cols[0]] && bcls[cols[1]] == bcls[cols[0]]),
              "job %zu: column blocks %d, %d", jx, cols[0], cols[1]);
        const bool same = bcls[rows[0]] == bcls[cols[0]];
        CHECK(same == ((int)jx < L.n_same), "job %zu: class order", jx);
        for (int r : rows)
            for (int c : cols)
                if (r >= 0 && c >= 0) cover[(size_t)r * nblk + c]++;
        // K trimming: nothing but vanishing terms outside [kb0, kb1)
        CHECK(j.kb0 >= 0 && j.kb0 <= j.kb1 && j.kb1 <= nblk, "job %zu: K [%d, %d) of %d", jx, j.kb0, j.kb1, nblk);
        int rmin = n, cmax = -1;
        for (int r : rows)
            for (int q = r * 64; r >= 0 && q < r * 64 + 64; q++)
                if (L.ginv[q] >= 0) rmin = std::min(rmin, L.ginv[q]);
        for (int c : cols)
            for (int q = c * 64; c >= 0 && q < c * 64 + 64; q++)
                if (L.ginv[q] >= 0) cmax = std::max(cmax, L.ginv[q]);
        for (int q = 0; q < L.ng; q++) {
            if (q >= j.kb0 * 64 && q < j.kb1 * 64) continue;
            const int k = L.ginv[q];
            g_checked++;
            CHECK(k < 0 || k <= rmin || k >= cmax, "job %zu: term k = %d (gathered %d) dropped, rows from %d, columns to %d",
                  jx, k, q, rmin, cmax);
        }
        const double used = (double)((rows[1] >= 0) + 1) * ((cols[1] >= 0) + 1) * (j.kb1 - j.kb0);
        (same ? kb_same : kb_opp) += used;
    }
    for (int r = 0; r < nblk; r++)
        for (int c = 0; c < nblk; c++) {
            const int want = bsb[r] <= bsb[c] ? 1 : 0;
            CHECK(cover[(size_t)r * nblk + c] == want, "blocks (%d, %d) in %d jobs, expected %d", r, c,
                  cover[(size_t)r * nblk + c], want);
        }
    CHECK(kb_same == L.kb_same && kb_opp == L.kb_opp, "K-block sums %g %g vs %g %g", kb_same, kb_opp, L.kb_same,
          L.kb_opp);
}

int main()
{
    std::mt19937 rng(20240607);
    const int sizes[] = {1, 2, 3, 63, 64, 65, 127, 128, 129, 200, 777, 1023, 1024, 1025, 1100, 2047, 2048, 2049,
                         3000, 4096, 5000, 8191, 16384};
    for (int n : sizes) {
        g_n = n;
        for (int kind = 0; kind < 9; kind++) {
            g_case = kind;
            if (n >= 8191 && kind % 3 != 0) continue;   // the large sizes: random, sorted, reversed
            std::vector<unsigned char> pos(n);
            const double p = (kind % 3 == 0) ? 0.5 : (kind % 3 == 1 ? 0.1 : 0.9);
            for (int i = 0; i < n; i++) pos[i] = std::uniform_real_distribution<double>(0, 1)(rng) >= p;
            if (kind >= 3 && kind < 6) std::sort(pos.begin(), pos.end(), [](int a, int b) { return a > b; });
            if (kind >= 6) std::sort(pos.begin(), pos.end());
            check(n, pos);
        }
        // one sign only, and alternating signs
        g_case = 9;
        check(n, std::vector<unsigned char>(n, 1));
        g_case = 10;
        check(n, std::vector<unsigned char>(n, 0));
        g_case = 11;
        std::vector<unsigned char> alt(n);
        for (int i = 0; i < n; i++) alt[i] = i & 1;
        check(n, alt);
    }
    if (g_fails) {
        std::printf("%d violations\n", g_fails);
        return 1;
    }
    std::printf("ok %lld\n", g_checked);
    return 0;
}

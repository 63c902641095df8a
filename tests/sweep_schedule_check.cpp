// Invariants of the tensor-core sweeps' work lists (sweep_schedule.h), for
// every tile count nb in [1, nb_max] (the lists depend on n only through nb):
//   - every tile (I, I+d) of a block anti-diagonal gets the block sums of
//     its K-blocks I .. I+d (Section 5.2: blocks strictly between, plus the
//     diagonal blocks' known in-block terms) exactly once -- from the plain
//     list, or, with look-ahead pairing, from the lead list at a lead
//     anti-diagonal and from look-ahead + completion lists at the next one;
//   - the look-ahead sums use only K-blocks whose blocks U(I,k), U(k,J) lie
//     on anti-diagonals solved before the lead one;
//   - CTA c writes its partial for tile t to slot c + t (2t, 2t+1 in the
//     completion), no slot twice, every slot below the list's max_jobs, and
//     each tile's (first, count) names exactly its slots, in K order;
//   - the look-ahead split is matched CTA by CTA to the lead one (same tile,
//     K-blocks inside the lead CTA's range);
//   - list sizes stay inside the workspace bounds the library reserves.
// Prints "ok <jobs checked>" and exits 0, or prints the first violations
// and exits 1.  Test infrastructure: compiled and run by the CPU tests.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "sweep_schedule.h"

using namespace signtri;

static int g_nb = 0;
static int g_fails = 0;
static long long g_jobs = 0;

#define CHECK(cond, ...)                                           \
    do {                                                           \
        if (!(cond)) {                                             \
            if (g_fails++ < 20) {                                  \
                std::printf("FAIL nb=%d line %d: ", g_nb, __LINE__); \
                std::printf(__VA_ARGS__);                          \
                std::printf("\n");                                 \
            }                                                      \
        }                                                          \
    } while (0)

struct Span {
    int j0, j1;  // jobs [j0, j1)
    int c0;      // first cta_off entry
    int t0;      // first tslot entry
};

static Span span_of(const Schedule &sc, int d)
{
    Span s;
    s.j0 = sc.job_off[d];
    s.j1 = d < sc.nb ? sc.job_off[d + 1] : (int)sc.jobs.size();
    s.c0 = sc.cta_begin[d];
    s.t0 = sc.tile_begin[d];
    return s;
}

// The CTA of each job of anti-diagonal d (from the per-CTA ranges; -1 for
// a job in no range).
static std::vector<int> ctas_of(const Schedule &sc, const Span &s, int d)
{
    std::vector<int> cta(s.j1 - s.j0, -1);
    for (int c = 0; c < sc.nctas[d]; c++)
        for (int q = sc.cta_off[s.c0 + c]; q < sc.cta_off[s.c0 + c + 1]; q++)
            if (q >= 0 && q < (int)cta.size()) cta[q] = c;
    return cta;
}

// Checks one list at anti-diagonal d.  cover[t][o] counts how often K-block
// I+o of tile t was summed (added to by this call).  `completion`: slots 2t
// and 2t+1 instead of c + t.  `nonempty`: every CTA has at least one job.
static void check_list(const Schedule &sc, int d, bool completion, bool nonempty,
                       std::vector<std::vector<int>> &cover)
{
    const int nb = sc.nb, ntiles = nb - d;
    const Span s = span_of(sc, d);
    const int G = sc.nctas[d];
    if (s.j1 == s.j0) {
        CHECK(G == 0, "d=%d: %d CTAs, no jobs", d, G);
        return;
    }
    CHECK(G >= 1 && G <= kSweepCtas, "d=%d: %d CTAs", d, G);
    CHECK(sc.cta_off[s.c0] == 0, "d=%d: first CTA range starts at %d", d, sc.cta_off[s.c0]);
    CHECK(sc.cta_off[s.c0 + G] == s.j1 - s.j0, "d=%d: CTA ranges end at %d of %d jobs", d, sc.cta_off[s.c0 + G],
          s.j1 - s.j0);
    for (int c = 0; c < G; c++) {
        const int a = sc.cta_off[s.c0 + c], b = sc.cta_off[s.c0 + c + 1];
        CHECK(a <= b, "d=%d: CTA %d range [%d, %d)", d, c, a, b);
        if (nonempty) CHECK(a < b, "d=%d: CTA %d empty", d, c);
    }
    const std::vector<int> cta = ctas_of(sc, s, d);
    std::vector<int> slot_tile(sc.max_jobs > 0 ? sc.max_jobs : 1, -1);
    std::vector<int> slot_k0(slot_tile.size(), -1);
    for (int j = s.j0; j < s.j1; j++) {
        const TcJob &jb = sc.jobs[j];
        g_jobs++;
        const int I = jb.rt / kSweepTile, J = jb.cl / kSweepTile;
        CHECK(jb.rt % kSweepTile == 0 && jb.cl % kSweepTile == 0, "d=%d job %d: rows %d cols %d", d, j, jb.rt, jb.cl);
        CHECK(jb.rb == jb.rt && jb.cr == jb.cl, "d=%d job %d: panels differ", d, j);
        CHECK(J - I == d && I >= 0 && I < ntiles, "d=%d job %d: tile (%d, %d)", d, j, I, J);
        CHECK(jb.kb0 < jb.kb1 && jb.kb0 >= I && jb.kb1 <= J + 1, "d=%d job %d: K [%d, %d) for tile (%d, %d)", d, j,
              jb.kb0, jb.kb1, I, J);
        if (!(I >= 0 && I < ntiles && jb.kb0 >= I && jb.kb1 <= J + 1)) continue;
        for (int k = jb.kb0; k < jb.kb1; k++) cover[I][k - I]++;
        const int c = cta[j - s.j0];
        CHECK(c >= 0, "d=%d job %d: in no CTA range", d, j);
        if (completion) {
            CHECK(jb.slot == 2 * I || jb.slot == 2 * I + 1, "d=%d job %d: slot %d for tile %d", d, j, jb.slot, I);
        } else {
            CHECK(jb.slot == c + I, "d=%d job %d: slot %d, CTA %d tile %d", d, j, jb.slot, c, I);
        }
        CHECK(jb.slot >= 0 && jb.slot < sc.max_jobs, "d=%d job %d: slot %d of %d", d, j, jb.slot, sc.max_jobs);
        if (jb.slot < 0 || jb.slot >= sc.max_jobs) continue;
        CHECK(slot_tile[jb.slot] < 0, "d=%d: slot %d written twice", d, jb.slot);
        slot_tile[jb.slot] = I;
        slot_k0[jb.slot] = jb.kb0;
    }
    // each tile's slot list: exactly its slots, K ascending
    int listed = 0;
    for (int t = 0; t < ntiles; t++) {
        const int2 ts = sc.tslot[s.t0 + t];
        int prev = -1;
        for (int q = ts.x; q < ts.x + ts.y; q++) {
            CHECK(q >= 0 && q < sc.max_jobs && slot_tile[q] == t, "d=%d tile %d: slot %d not its own", d, t, q);
            if (q < 0 || q >= sc.max_jobs) continue;
            CHECK(slot_k0[q] > prev, "d=%d tile %d: slots out of K order", d, t);
            prev = slot_k0[q];
        }
        listed += ts.y;
        // a full split (one sweep launch) gives a tile at most kMaxSlotsPerTile
        // CTAs, so at most that many slots plus one per CTA-range boundary
        CHECK(ts.y <= kMaxSlotsPerTile + 1, "d=%d tile %d: %d slots", d, t, ts.y);
    }
    CHECK(listed == s.j1 - s.j0, "d=%d: %d slots listed for %d jobs", d, listed, s.j1 - s.j0);
}

// B's CTA c sums, for each of its tiles, K-blocks inside lead CTA c's range
// of the same tile (the two launches read the same row panels together).
static void check_matched(const Schedule &A, int dl, const Schedule &B, int e)
{
    const Span sa = span_of(A, dl), sb = span_of(B, e);
    CHECK(A.nctas[dl] == B.nctas[e], "e=%d: %d look-ahead CTAs vs %d lead CTAs", e, B.nctas[e], A.nctas[dl]);
    const std::vector<int> cta = ctas_of(B, sb, e);
    for (int j = sb.j0; j < sb.j1; j++) {
        const TcJob &jb = B.jobs[j];
        const int c = cta[j - sb.j0], I = jb.rt / kSweepTile;
        CHECK(c >= 0 && c < A.nctas[dl], "e=%d job %d: CTA %d", e, j, c);
        if (c < 0 || c >= A.nctas[dl]) continue;
        bool inside = false;
        for (int q = sa.j0 + A.cta_off[sa.c0 + c]; q < sa.j0 + A.cta_off[sa.c0 + c + 1]; q++) {
            const TcJob &ja = A.jobs[q];
            if (ja.rt == jb.rt && jb.kb0 - I >= ja.kb0 - I && jb.kb1 - I <= ja.kb1 - I) inside = true;
        }
        CHECK(inside, "e=%d job %d (tile %d, K [%d, %d)): outside lead CTA %d's range", e, j, I, jb.kb0, jb.kb1, c);
    }
}

static void check_bounds(const Schedule &sc, const char *what)
{
    const long long nb = sc.nb;
    CHECK(sc.max_jobs <= kSweepCtas + 2 * nb + 8, "%s: max_jobs %d", what, sc.max_jobs);
    CHECK((long long)sc.jobs.size() <= nb * (kSweepCtas + 2 * nb), "%s: %zu jobs", what, sc.jobs.size());
    CHECK((long long)sc.cta_off.size() <= nb * (kSweepCtas + 1), "%s: %zu CTA entries", what, sc.cta_off.size());
    CHECK((long long)sc.tslot.size() <= nb * nb, "%s: %zu tile entries", what, sc.tslot.size());
}

static std::vector<std::vector<int>> zero_cover(int nb, int d)
{
    return std::vector<std::vector<int>>(nb - d, std::vector<int>(d + 1, 0));
}

static void check_nb(int nb)
{
    g_nb = nb;
    const int n = nb * kSweepTile;
    for (int gmax : {kSweepCtas, kSweepCtas / 2}) {
        Schedule sc;
        build_schedule(n - (nb > 1 ? 17 : 0), gmax, sc);  // a ragged n with the same tile count
        CHECK(sc.nb == nb, "plain list for %d tiles has nb %d", nb, sc.nb);
        for (int d = 0; d <= nb; d++) {
            if (d == 0 || d == nb) {
                CHECK(span_of(sc, d).j0 == span_of(sc, d).j1, "d=%d: jobs on an empty anti-diagonal", d);
                continue;
            }
            auto cover = zero_cover(nb, d);
            check_list(sc, d, false, true, cover);
            for (int t = 0; t < nb - d; t++)
                for (int o = 0; o <= d; o++) CHECK(cover[t][o] == 1, "plain d=%d tile %d K-block +%d summed %d times", d, t, o, cover[t][o]);
        }
        check_bounds(sc, "plain");
    }
    for (int gmax : {kSweepCtas / 2, kSweepCtas}) {
        Schedule A, B, C, P;
        build_look_schedules(n, gmax, A, B, C);
        build_schedule(n, gmax, P);
        for (int d = 1; d < nb; d++) {
            const bool lead = look_lead(d, nb), follow = look_follow(d, nb);
            CHECK(!(lead && follow), "d=%d both lead and follow", d);
            if (lead) CHECK(look_follow(d + 1, nb), "lead d=%d without a follow", d);
            auto cover = zero_cover(nb, d);
            check_list(A, d, false, true, cover);
            if (lead) {
                // the lead list is the plain split of d
                const Span sa = span_of(A, d), sp = span_of(P, d);
                CHECK(sa.j1 - sa.j0 == sp.j1 - sp.j0, "lead d=%d: %d jobs vs plain %d", d, sa.j1 - sa.j0, sp.j1 - sp.j0);
            } else {
                CHECK(span_of(A, d).j0 == span_of(A, d).j1, "d=%d: lead jobs off a lead anti-diagonal", d);
            }
            if (follow) {
                auto look = zero_cover(nb, d);
                check_list(B, d, false, false, look);
                // look-ahead K-blocks only from anti-diagonals before the lead one
                for (int t = 0; t < nb - d; t++)
                    for (int o = 0; o <= d; o++)
                        if (look[t][o]) CHECK(o >= 2 && d - o >= 2, "follow d=%d tile %d: K-block +%d needs the lead anti-diagonal", d, t, o);
                check_list(C, d, true, true, cover);
                for (int t = 0; t < nb - d; t++)
                    for (int o = 0; o <= d; o++) cover[t][o] += look[t][o];
                check_matched(A, d - 1, B, d);
            } else {
                CHECK(span_of(B, d).j0 == span_of(B, d).j1, "d=%d: look-ahead jobs off a follow anti-diagonal", d);
                CHECK(span_of(C, d).j0 == span_of(C, d).j1, "d=%d: completion jobs off a follow anti-diagonal", d);
            }
            if (lead || follow) {
                for (int t = 0; t < nb - d; t++)
                    for (int o = 0; o <= d; o++)
                        CHECK(cover[t][o] == 1, "paired d=%d tile %d K-block +%d summed %d times", d, t, o, cover[t][o]);
            }
        }
        check_bounds(A, "lead");
        check_bounds(B, "look-ahead");
        check_bounds(C, "completion");
    }
}

// Arguments: every tile count 1 .. argv[1] (default 200), then each further
// argument as one more tile count.
int main(int argc, char **argv)
{
    const int nb_max = argc > 1 ? std::atoi(argv[1]) : 200;
    for (int nb = 1; nb <= nb_max; nb++) check_nb(nb);
    for (int a = 2; a < argc; a++) check_nb(std::atoi(argv[a]));
    if (g_fails) {
        std::printf("%d violations\n", g_fails);
        return 1;
    }
    std::printf("ok %lld\n", g_jobs);
    return 0;
}

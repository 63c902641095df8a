// sweep_schedule.h -- host-side work lists of the tensor-core block-sum
// sweeps of the mixed variants (mixed.cu): which CTA sums which K-blocks of
// which tile of an anti-diagonal, into which partial slot, and which slots
// each tile's leaf adds up (Section 5.2's block sums X, Y of the tiles of one
// block anti-diagonal, cut into equal CTA ranges).  Host code only; the
// tests compile it on its own to check the work lists' invariants.
#pragma once

#include <vector_types.h>

#include <algorithm>
#include <vector>

#include "tc_job.h"

namespace signtri {

// Rows and columns of a tile, and the width of a K-block.
constexpr int kSweepTile = 64;

// Block sums of one anti-diagonal, split evenly over G persistent CTAs (the
// tiles' K-blocks in a row, cut into equal ranges; a CTA's range may cross
// tile boundaries): CTA c's partial for tile t goes to slot c + t, and tile
// t's partials are the slots first(t)+t .. last(t)+t (in K order).  The
// initial sweep's single launch per anti-diagonal takes kSweepCtas CTAs; the
// correction's two launches run side by side with half as many each, on the
// same split, so that the CTA pairs that read the same E panels at the same
// time share them through L2.
constexpr int kSweepCtas = 152;
// At most this many CTAs (partial slots) per tile: the leaf adds a tile's
// slots one after another, so on the last anti-diagonals, where few tiles
// would share all CTAs, a longer K range per CTA costs less than the slots.
constexpr int kMaxSlotsPerTile = 16;

inline int sweep_ctas(int gmax, int ntiles, long long W)
{
    return (int)std::min<long long>(std::min<long long>(gmax, W), (long long)ntiles * kMaxSlotsPerTile);
}

struct Schedule {
    int nb = 0;
    std::vector<int> job_off;   // per anti-diagonal d: first job index (d = 0..nb)
    std::vector<int> cta_off;   // concatenated per-diagonal CTA job ranges (local indices)
    std::vector<int> cta_begin; // per d: first entry in cta_off
    std::vector<int> nctas;     // per d: CTAs of the block-sum launch (0: none)
    std::vector<int2> tslot;    // concatenated per-tile (first slot, count)
    std::vector<int> tile_begin;// per d: first entry in tslot
    std::vector<TcJob> jobs;
    int max_jobs = 0;           // partial slots needed by one diagonal
};

inline void schedule_reset(int nb, Schedule &sc)
{
    sc.nb = nb;
    sc.job_off.assign(nb + 1, 0);
    sc.cta_begin.assign(nb + 1, 0);
    sc.nctas.assign(nb + 1, 0);
    sc.tile_begin.assign(nb + 1, 0);
    sc.cta_off.clear();
    sc.tslot.clear();
    sc.jobs.clear();
    sc.max_jobs = 0;
}

// Marks where anti-diagonal d's entries begin (call for d = 0 .. nb in order).
inline void schedule_open(Schedule &sc, int d)
{
    sc.job_off[d] = (int)sc.jobs.size();
    sc.cta_begin[d] = (int)sc.cta_off.size();
    sc.tile_begin[d] = (int)sc.tslot.size();
}

inline TcJob tile_job(int I, int J, int kb0, int kb1, int slot)
{
    TcJob j;
    j.rt = I * kSweepTile; j.rb = I * kSweepTile; j.cl = J * kSweepTile; j.cr = J * kSweepTile;
    j.kb0 = kb0; j.kb1 = kb1; j.slot = slot; j.pad = 0;
    return j;
}

// The full block sums of anti-diagonal d (K-blocks I .. J: the diagonal
// blocks carry the known in-block terms), split evenly over up to gmax CTAs.
inline void add_even_split(Schedule &sc, int d, int nb, int gmax)
{
    const int ntiles = nb - d;
    const long long kmax = d + 1, W = (long long)ntiles * kmax;
    const int G = sweep_ctas(gmax, ntiles, W);
    sc.nctas[d] = G;
    const int base = (int)sc.jobs.size();
    for (int c = 0; c < G; c++) {
        sc.cta_off.push_back((int)sc.jobs.size() - base);
        const long long x1 = (long long)(c + 1) * W / G;
        for (long long x = (long long)c * W / G; x < x1;) {
            const int t = (int)(x / kmax);
            const long long t0 = (long long)t * kmax, xe = std::min(x1, t0 + kmax);
            sc.jobs.push_back(tile_job(t, t + d, t + (int)(x - t0), t + (int)(xe - t0), c + t));
            x = xe;
        }
    }
    sc.cta_off.push_back((int)sc.jobs.size() - base);
    for (int t = 0; t < ntiles; t++) {
        // the CTA holding chunk x is ((x + 1) G - 1) / W (every CTA's range is non-empty)
        const long long f = (((long long)t * kmax + 1) * G - 1) / W;
        const long long l = (((long long)(t + 1) * kmax) * G - 1) / W;
        sc.tslot.push_back(int2{(int)(f + t), (int)(l - f + 1)});
    }
    sc.max_jobs = std::max(sc.max_jobs, G + ntiles);
}

inline void build_schedule(int n, int gmax, Schedule &sc)
{
    const int nb = (n + kSweepTile - 1) / kSweepTile;
    schedule_reset(nb, sc);
    for (int d = 0; d <= nb; d++) {
        schedule_open(sc, d);
        if (d >= 1 && d < nb) add_even_split(sc, d, nb, gmax);
    }
}

// Look-ahead pairing of the initial sweep: for a lead anti-diagonal d (odd,
// >= 3, with d + 1 < nb), the tiles (I, I+d+1) of the next one take their
// block sums over K-blocks I+2 .. I+d-1 -- all known before anti-diagonal d
// is solved -- in a launch that runs beside d's own, on a split matched CTA
// by CTA to d's: CTA c of both walks the same row panels I at the same
// K-blocks, so the look-ahead reads them from L2.  The four K-blocks left,
// I, I+1, I+d, I+d+1 (two of them involve anti-diagonal d), are summed
// after d's leaves by a completion launch.
inline bool look_lead(int d, int nb) { return d >= 3 && (d & 1) && d + 1 < nb; }
inline bool look_follow(int d, int nb) { return d >= 4 && !(d & 1) && look_lead(d - 1, nb); }

inline void build_look_schedules(int n, int gmax, Schedule &A, Schedule &B, Schedule &C)
{
    const int nb = (n + kSweepTile - 1) / kSweepTile;
    schedule_reset(nb, A);
    schedule_reset(nb, B);
    schedule_reset(nb, C);
    for (int d = 0; d <= nb; d++) {
        schedule_open(A, d);
        schedule_open(B, d);
        schedule_open(C, d);
        if (d < 1 || d >= nb) continue;
        if (look_lead(d, nb)) add_even_split(A, d, nb, gmax);
        if (!look_follow(d, nb)) continue;
        // B: the look-ahead sums of anti-diagonal e = d, matched to A's split of d - 1
        const int e = d, dl = d - 1, nl = nb - dl, ne = nb - e;
        const long long kmax = dl + 1, W = (long long)nl * kmax;
        const int G = sweep_ctas(gmax, nl, W);   // the lead's split
        B.nctas[e] = G;
        const int base = (int)B.jobs.size();
        for (int c = 0; c < G; c++) {
            B.cta_off.push_back((int)B.jobs.size() - base);
            const long long x0 = (long long)c * W / G, x1 = (long long)(c + 1) * W / G;
            for (int t = (int)(x0 / kmax); t <= (int)((x1 - 1) / kmax) && t < ne; t++) {
                const long long lo = std::max<long long>(x0 - (long long)t * kmax, 2);
                const long long hi = std::min<long long>(x1 - (long long)t * kmax, dl);   // offsets 2 .. dl-1
                if (lo < hi) B.jobs.push_back(tile_job(t, t + e, t + (int)lo, t + (int)hi, c + t));
            }
        }
        B.cta_off.push_back((int)B.jobs.size() - base);
        for (int t = 0; t < ne; t++) {
            const long long f = (((long long)t * kmax + 2 + 1) * G - 1) / W;
            const long long l = (((long long)t * kmax + dl - 1 + 1) * G - 1) / W;
            B.tslot.push_back(int2{(int)(f + t), (int)(l - f + 1)});
        }
        B.max_jobs = std::max(B.max_jobs, G + nl);
        // C: the completion, K-blocks I, I+1 and I+e-1, I+e of every tile, two slots a tile
        const int GC = std::min(kSweepCtas, ne);
        C.nctas[e] = GC;
        const int cbase = (int)C.jobs.size();
        for (int c = 0; c < GC; c++) {
            C.cta_off.push_back((int)C.jobs.size() - cbase);
            for (int t = (int)((long long)c * ne / GC); t < (int)((long long)(c + 1) * ne / GC); t++) {
                C.jobs.push_back(tile_job(t, t + e, t, t + 2, 2 * t));
                C.jobs.push_back(tile_job(t, t + e, t + e - 1, t + e + 1, 2 * t + 1));
            }
        }
        C.cta_off.push_back((int)C.jobs.size() - cbase);
        for (int t = 0; t < ne; t++) C.tslot.push_back(int2{2 * t, 2});
        C.max_jobs = std::max(C.max_jobs, 2 * ne);
    }
}

}  // namespace signtri

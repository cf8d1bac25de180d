// Group-per-walker Wang-Landau sampling with tree speculation (sm_103a).
//
// The trials of one walker form a sequential Markov chain (Eq. 1 and the
// update rule of Sec. 2 of arXiv:1508.02748): each trial depends on the
// accept/reject outcome of the one before.  A group of G lanes (G = 8, 16 or
// 32; 32/G walkers per warp) runs one walker and resolves DEPTH+1 trials per
// step (DEPTH = log2(G) - 1): lanes 0..G-2 form a binary tree; lane l sits at
// depth d = floor(log2(l+1)) and evaluates trial t+d under the history
// h = l + 1 - 2^d (bit k of h = outcome assumed for trial t+k).
//
// Per step every lane
//   1. reads its own trial's site from the ring and the five spins around it
//      from the committed lattice, corrected for the sites its history flips;
//      this gives the move (de, dm) of its trial under its history;
//   2. takes the moves of the earlier trials of its history by shuffle from
//      the lanes that evaluated them (lane 2^k - 1 + (h mod 2^k) for trial k),
//      and walks them to find its current bin and the bins visited;
//   3. decides its own trial (Eq. 1) with the exact ln g values the sequential
//      chain would see there: value(bin) = table(bin) + visits * ln f.
// One ballot gives the true path from the root: a lane is on it iff the
// ballot bits of its ancestors are the outcomes its history assumes.  Lane k
// of the path knows the bin the walker is in after trial t+k and posts it in
// a per-walker mailbox in shared memory; after one warp barrier every lane
// knows the path's bins, the leaf's (E, M) and its flips, and lane k commits
// trial k: its spin flip, and the ln g / H update of its bin if that bin is
// left in this step (first occurrence only, with all its visits).
//
// Tables staged in shared memory (double or compensated pairs) are not
// updated during a launch: H counts the launch's visits Q(b), a bin's value
// is table(b) + Q(b) ln f, and the counts are folded into the tables when
// the launch writes them back.  The float screen reads a 32-bit copy of each
// staged value.
//
// The outcome is the sequential chain itself, trial for trial:
//   - random numbers are drawn per trial index from the TRIAL stream of
//     Philox4x32-10, independent of the state (a ring of 128 trials per
//     walker, refilled 64 at a time from the even trial at or below the
//     launch's first trial);
//   - table(bin) + visits * ln f is evaluated exactly: fma in double for
//     REWL_FP64, a compensated (hi, lo) float sum for REWL_F32X2; both equal
//     the sequential additions whenever ln f = 2^-k and the values stay
//     within the exact range of the format;
//   - decisions are screened in float with a margin that bounds the float
//     rounding (|x - float(x)| < 2^-23 |x| for both table formats) and
//     re-taken exactly on near-ties (out of line: the exact difference
//     against the float ln u, and ln u in double only when those two are
//     within 2^-20 (|ln u| + 1)).
// The walker's current bin stays in registers (its table value at entry,
// the visits since then) and is written back when the walker leaves it.
#include "rewl_tab.cuh"

namespace rewl {

using namespace tab;

namespace {

constexpr int RING = 128;   // trials buffered per walker

// One buffered trial (16 bytes, one shared-memory vector load).  Everything
// about a trial that does not depend on the walker's state is computed when
// the ring is refilled: the site and its four periodic neighbours, and ln u.
struct RingEntry {
    uint32_t a;    // register lattice: the 6-bit indices of the site and of its up,
                   //   down, left and right neighbours at bits 0, 6, 12, 18, 24;
                   // shared lattice: row | col << 8 | up-row << 16 | down-row << 24
    uint32_t b;    // shared lattice: left-col | right-col << 8
    uint32_t xu;   // acceptance word
    float lnu;     // ln u in float
};

// Per-walker exchange area of one step (shared memory): the lanes of a
// group trade their trial results through it instead of warp shuffles.
struct Mailbox {
    int dummy[32];                 // discarded stores of the branch-free write-back
    int after[8];                  // bin after trial t+k on the true path
    int leafpos;                   // the leaf's new (e, m)
    int pad;
    unsigned long long flips;      // register lattice: the path's flip mask
};

// Eq. 1 decided from the exact values (near-ties of the float screen only);
// kept out of line so none of it runs in the common case.  The difference
// delta is exact in double.  The float ln u of the ring (logf of u rounded to
// float) is within 2^-22 (|ln u| + 1) of ln u: u rounds with relative error
// below 2^-23 and logf errs by at most 1 ulp (its documented bound).  So
// outside a band 4x wider the float ln u decides, and only inside it is ln u
// taken in double (the double logarithm is slow here).
template <class TB>
__device__ __noinline__ int exact_accept(typename TB::Val cbase, int ccnt, typename TB::Val nbase, int ncnt,
                                         double lnf, uint32_t xu, float lnu32)
{
    const double delta = fma((double)ccnt, lnf, TB::exact(cbase)) - fma((double)ncnt, lnf, TB::exact(nbase));
    if (delta >= 0.0) return 1;
    const double lu = (double)lnu32;
    const double band = (fabs(lu) + 1.0) * 0x1p-20;
    if (lu < delta - band) return 1;
    if (lu > delta + band) return 0;
    return log(unit_open_d(xu)) < delta ? 1 : 0;
}

// The same with staged tables that keep their launch-start values: the base
// values are read from the staged table here, off the common path.
template <class TB>
__device__ __noinline__ int exact_accept_staged(const typename TB::Elem *tl, int cb, int ccnt, int nb, int ncnt,
                                                double lnf, uint32_t xu, float lnu32)
{
    return exact_accept<TB>(TB::load(tl, cb), ccnt, TB::load(tl, nb), ncnt, lnf, xu, lnu32);
}

template <int G>
struct TreeShape {
    static constexpr int DEPTH = G == 32 ? 4 : G == 16 ? 3 : G == 8 ? 2 : 1;
};

}  // namespace

// REG: the lattice (N <= 64 sites, bit i*L + j) is held in a 64-bit register
// by every lane; otherwise it lives in shared memory, one 32-bit word per row
// (two for L > 32).
template <int WPR, bool SMT, int G, int PREC, bool REG>
__global__ void __launch_bounds__(256) k_sweep_tree(Params p, unsigned ntrials, int smem_per_walker)
{
    using TB = Tab<PREC>;
    using Elem = typename TB::Elem;
    using Val = typename TB::Val;
    constexpr int DEPTH = TreeShape<G>::DEPTH;
    // LAZY (tables staged in shared memory, exact formats): the staged ln g
    // values stay those of the launch start and the shared H array counts the
    // visits of this launch, Q(b); the value of bin b is table(b) + Q(b) ln f,
    // folded into the tables once, when they are written back.  No
    // floating-point update runs per trial (the double update is slow here).
    constexpr bool LAZY = SMT && PREC != REWL_F32;
    constexpr int GPW = 32 / G;   // walkers per warp
    constexpr unsigned GBITS = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane & (G - 1), grp = lane / G;
    const unsigned gmask = GBITS << (grp * G);
    const int slot = wid * GPW + grp;   // walker slot within the block
    const int w = blockIdx.x * ((blockDim.x >> 5) * GPW) + slot;
    if (w >= p.nwalk) return;
    if (!p.active[w / p.W] || p.st->done) return;

    unsigned char *base = smem_raw + (size_t)slot * smem_per_walker;
    RingEntry *ring = reinterpret_cast<RingEntry *>(base);
    Mailbox *box = reinterpret_cast<Mailbox *>(base + RING * sizeof(RingEntry));
    uint32_t *lat = reinterpret_cast<uint32_t *>(base + RING * sizeof(RingEntry) + sizeof(Mailbox));
    const int L = p.L, nwords = L * WPR;
    const int T = p.T;
    Elem *g_tab = (PREC == REWL_FP64) ? reinterpret_cast<Elem *>(p.lng)
                : (PREC == REWL_F32X2) ? reinterpret_cast<Elem *>(p.lng2) : reinterpret_cast<Elem *>(p.lng1);
    g_tab += (size_t)w * p.tstride;
    int32_t *gH = p.H + (size_t)w * p.tstride;
    Elem *tl;
    int32_t *tH;
    if (SMT) {
        tl = reinterpret_cast<Elem *>(base + RING * sizeof(RingEntry) + sizeof(Mailbox) + ((nwords * 4 + 15) & ~15));
        tH = reinterpret_cast<int32_t *>(tl + T);
        for (int k = gl; k < T; k += G) { tl[k] = g_tab[k]; tH[k] = LAZY ? 0 : gH[k]; }
        if constexpr (LAZY && PREC == REWL_FP64) {
            float *t32 = reinterpret_cast<float *>(tH + T);
            for (int k = gl; k < T; k += G) t32[k] = TB::approx(g_tab[k]);
        }
    } else {
        tl = g_tab;
        tH = gH;
    }
    unsigned long long lat64 = 0;
    if (REG) {
        for (int r = 0; r < L; ++r)
            lat64 |= (unsigned long long)p.spins[(size_t)r * p.nwalk + w] << (r * L);
    } else {
        for (int k = gl; k < nwords; k += G) lat[k] = p.spins[(size_t)k * p.nwalk + w];
    }
    __syncwarp(gmask);

    const int4 R = p.rect[w / p.W];
    const int wM = p.wM;
    const unsigned spanE = (unsigned)(R.y - R.x), spanM = (unsigned)(R.w - R.z);
    const double lnf = p.st->lnf;
    const float lnf32 = trunc_f(lnf);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t divL = p.divL;

    // this lane's node of the tree and the lanes holding its history's trials
    const int dl = 31 - __clz(gl + 1);
    const int hist = gl + 1 - (1 << dl);
    int srck[DEPTH];
    #pragma unroll
    for (int k = 0; k < DEPTH; ++k) srck[k] = (1 << k) - 1 + (hist & ((1 << k) - 1));
    // the lane is on the true path iff the ballot bits of its ancestors
    // (lane 2^k - 1 + (h mod 2^k) at depth k < d) are the outcomes its
    // history assumes: anc marks the ancestors, want holds those outcomes
    unsigned anc = 0, want = 0;
    #pragma unroll
    for (int k = 0; k <= DEPTH; ++k)
        if (k < dl) {
            const int a = (1 << k) - 1 + (hist & ((1 << k) - 1));
            anc |= 1u << a;
            want |= (unsigned)((hist >> k) & 1) << a;
        }

    // committed state (uniform over the group)
    int e = p.we[w], m = p.wm[w];
    int ci = (e - R.x) * wM + (m - R.z);
    // LAZY: the float screen reads one 32-bit word per bin: the float copy of
    // a double table (staged after H), the hi word of a compensated pair
    const float *scr32 = !LAZY ? nullptr
                       : (PREC == REWL_FP64) ? reinterpret_cast<const float *>(tH + T)
                                             : reinterpret_cast<const float *>(tl);
    constexpr int SCR_STRIDE = PREC == REWL_FP64 ? 1 : 2;
    Val lbase = TB::load(tl, ci);   // table value of the current bin when entered
    int lq = 0;                     // ln f steps since lbase (LAZY: visits of this launch)
    int hq = 0;                     // visits of the current bin not yet in H (LAZY: in Q)
    int hbase = tH[ci];
    float base32 = TB::approx(lbase);
    const unsigned long long t0 = p.wt[w];
    const unsigned r0 = (unsigned)t0 & (RING - 1);
    unsigned u = 0;                 // trials done in this launch
    unsigned ufill = 0;             // ring holds trials [t0 - (t0 & 1), t0 + ufill)
    const unsigned long long c0 = t0 >> 1;   // first Philox call
    unsigned cfill = 0;             // calls done
    int err = 0;

    while (u < ntrials) {
        // ---- refill the ring: 32 Philox calls = 64 trials
        if (ufill < u + 32) {
            #pragma unroll
            for (int r = 0; r < 32 / G; ++r) {
                const unsigned long long c = c0 + cfill + (unsigned)(gl + r * G);
                const u32x4 x = philox10((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)w, TAG_TRIAL, p.key0, p.key1);
                #pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const uint32_t xs = hh ? x.z : x.x, xu = hh ? x.w : x.y;
                    const uint32_t site = __umulhi(xs, N);
                    const uint32_t i = __umulhi(site, divL);
                    const uint32_t j = site - i * (uint32_t)L;
                    const uint32_t iu = i == 0 ? L - 1 : i - 1, id = i == (uint32_t)L - 1 ? 0 : i + 1;
                    const uint32_t jl = j == 0 ? L - 1 : j - 1, jr = j == (uint32_t)L - 1 ? 0 : j + 1;
                    RingEntry en;
                    if (REG) {
                        en.a = site | ((iu * L + j) << 6) | ((id * L + j) << 12) | ((i * L + jl) << 18) | ((i * L + jr) << 24);
                        en.b = 0;
                    } else {
                        en.a = i | (j << 8) | (iu << 16) | (id << 24);
                        en.b = jl | (jr << 8);
                    }
                    en.xu = xu;
                    en.lnu = logf(__fmaf_rn(__uint2float_rn(xu), 0x1p-32f, 0x1p-33f));
                    ring[(unsigned)(2 * c + hh) & (RING - 1)] = en;
                }
            }
            cfill += 32;
            ufill = 2 * cfill - (unsigned)(t0 & 1ull);
            __syncwarp(gmask);
        }
        if (!LAZY && lq >= (1 << 22)) {   // keep the float screen's counts exact (LAZY
                                          // launches run fewer than 2^22 trials)
            lbase = TB::add(lbase, lq, lnf, lnf32);
            lq = 0;
            base32 = TB::approx(lbase);
        }
        const unsigned left = ntrials - u;
        const int D = left > (unsigned)DEPTH ? DEPTH : (int)left - 1;
        const unsigned rb = r0 + u;

        // ---- 1. own trial under own history
        const RingEntry me = ring[(rb + dl) & (RING - 1)];
        uint32_t sa[DEPTH + 1];      // site words of trials t .. t+DEPTH (uniform)
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) sa[k] = ring[(rb + k) & (RING - 1)].a;
        uint32_t sbit, bu, bd, bl, br;
        unsigned long long fm = 0;   // register lattice: sites flipped by the history
        if (REG) {
            #pragma unroll
            for (int k = 0; k < DEPTH; ++k)
                if (k < dl && ((hist >> k) & 1)) fm ^= 1ull << (sa[k] & 63u);   // a site may flip twice
            const unsigned long long v = lat64 ^ fm;
            sbit = (uint32_t)(v >> (me.a & 63u)) & 1u;
            bu = (uint32_t)(v >> ((me.a >> 6) & 63u)) & 1u;
            bd = (uint32_t)(v >> ((me.a >> 12) & 63u)) & 1u;
            bl = (uint32_t)(v >> ((me.a >> 18) & 63u)) & 1u;
            br = (uint32_t)(v >> ((me.a >> 24) & 63u)) & 1u;
        } else {
            const int i = me.a & 255, j = (me.a >> 8) & 255, iu = (me.a >> 16) & 255, id = me.a >> 24;
            const int jl = me.b & 255, jr = (me.b >> 8) & 255;
            const int qj = (WPR == 1) ? 0 : (j >> 5);
            const uint32_t wc = lat[i * WPR + qj], wu = lat[iu * WPR + qj], wd = lat[id * WPR + qj];
            sbit = (wc >> (j & 31)) & 1u;
            bu = (wu >> (j & 31)) & 1u;
            bd = (wd >> (j & 31)) & 1u;
            bl = ((WPR == 1 ? wc : lat[i * WPR + (jl >> 5)]) >> (jl & 31)) & 1u;
            br = ((WPR == 1 ? wc : lat[i * WPR + (jr >> 5)]) >> (jr & 31)) & 1u;
            const uint32_t p_s = i | (j << 8), p_u = iu | (j << 8), p_d = id | (j << 8);
            const uint32_t p_l = i | (jl << 8), p_r = i | (jr << 8);
            #pragma unroll
            for (int k = 0; k < DEPTH; ++k) {
                if (k < dl && ((hist >> k) & 1)) {
                    const uint32_t f = sa[k] & 0xFFFFu;
                    sbit ^= (f == p_s);
                    bu ^= (f == p_u);
                    bd ^= (f == p_d);
                    bl ^= (f == p_l);
                    br ^= (f == p_r);
                }
            }
        }
        const int nup = (int)(bu + bd + bl + br);
        const int de_own = sbit ? nup - 2 : 2 - nup;
        const int dm_own = sbit ? -1 : 1;
        const int pack = (de_own + 2) | ((dm_own + 1) << 3);

        // ---- 2. the history's earlier trials: the move of trial k under the
        // history's first k outcomes is the own move of lane 2^k - 1 + (h mod 2^k),
        // taken by shuffle; a history that accepts a move out of the window is
        // never the true path, and its bins are clamped below only to keep its
        // reads in bounds
        int ce = e, cm = m, cbin = ci;
        int vb[DEPTH];               // bin after each earlier trial (-1 past the own depth)
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            const int pk = __shfl_sync(gmask, pack, grp * G + srck[k]);
            if (k < dl && ((hist >> k) & 1)) {
                const int de = (pk & 7) - 2, dm = ((pk >> 3) & 3) - 1;
                ce += de;
                cm += dm;
                cbin += de * wM + dm;
            }
            vb[k] = k < dl ? cbin : -1;
        }

        // ---- 3. decision of the own trial (Eq. 1)
        const int en_o = ce + de_own, mn_o = cm + dm_own;
        const int nbin = cbin + de_own * wM + dm_own;
        const bool live = dl <= D && (unsigned)(en_o - R.x) <= spanE && (unsigned)(mn_o - R.z) <= spanM;
        const int cb = min(max(cbin, 0), T - 1), nb = min(max(nbin, 0), T - 1);
        int vcur = 0, vnew = 0;
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            vcur += (vb[k] == cb);
            vnew += (vb[k] == nb);
        }
        const bool c0b = cb == ci, n0b = nb == ci;
        Val cbase, nbase;
        float cb32, nb32;
        if constexpr (LAZY) {
            cb32 = c0b ? base32 : scr32[cb * SCR_STRIDE];
            nb32 = n0b ? base32 : scr32[nb * SCR_STRIDE];
        } else {
            const Val tc = TB::load(tl, cb), tn = TB::load(tl, nb);
            cbase = c0b ? lbase : tc;
            nbase = n0b ? lbase : tn;
            cb32 = c0b ? base32 : TB::approx(tc);
            nb32 = n0b ? base32 : TB::approx(tn);
        }
        const int qc = LAZY ? tH[cb] : 0, qn = LAZY ? tH[nb] : 0;
        const int ccnt = vcur + (c0b ? lq : qc), ncnt = vnew + (n0b ? lq : qn);
        const float c32 = __fmaf_rn((float)ccnt, lnf32, cb32);
        const float n32 = __fmaf_rn((float)ncnt, lnf32, nb32);
        const float d32 = c32 - n32;
        const float M = (fabsf(c32) + fabsf(n32) + fabsf(cb32) + fabsf(nb32) + fabsf(me.lnu)) * 0x1p-20f + 0x1p-20f;
        int acc = (me.lnu < d32 - M) ? 1 : 0;
        if constexpr (PREC == REWL_F32) {
            // plain float: the values the walker sees are the rounded sums
            acc = (me.lnu < TB::add(cbase, ccnt, lnf, lnf32) - TB::add(nbase, ncnt, lnf, lnf32)) ? 1 : 0;
        } else if (live && !acc && !(me.lnu > d32 + M)) {
            // LAZY: the current bin's base is its staged value too (lbase == tl[ci])
            if constexpr (LAZY) acc = exact_accept_staged<TB>(tl, cb, ccnt, nb, ncnt, lnf, me.xu, me.lnu);
            else acc = exact_accept<TB>(cbase, ccnt, nbase, ncnt, lnf, me.xu, me.lnu);
        }
        acc = live ? acc : 0;
        const int after = acc ? nbin : cbin;   // bin after the own trial, under the own history

        // ---- the true path: the lanes whose ancestors decided as their history assumes
        const unsigned bal = (__ballot_sync(gmask, acc) >> (grp * G)) & GBITS;
        const bool onp = dl <= D && ((bal ^ want) & anc) == 0u;
        const bool is_leaf = onp && dl == D;

        // ---- commit: the on-path lane of depth k takes trial t+k
        if (onp) box->after[dl] = after;
        if (is_leaf) {
            box->leafpos = ((acc ? en_o : ce) << 13) | (acc ? mn_o : cm);
            if (REG) box->flips = fm ^ (acc ? (1ull << (me.a & 63u)) : 0ull);
        }
        __syncwarp(gmask);
        int av[DEPTH + 1];
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) av[k] = k <= D ? box->after[k] : -1;
        const int lp = box->leafpos;
        const int ne = lp >> 13, nm = lp & 0x1FFF;
        const int C = (ne - R.x) * wM + (nm - R.z);
        int cC = 0;
        bool b0_seen = false;
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) {
            cC += (av[k] == C);
            b0_seen |= (av[k] == ci);
        }
        if (REG) {
            lat64 ^= box->flips;
        } else if (onp && acc) {
            const int fi = me.a & 255, fj = (me.a >> 8) & 255;
            atomicXor(&lat[fi * WPR + ((WPR == 1) ? 0 : (fj >> 5))], 1u << (fj & 31));
        }
        // first visit of this lane's bin among the path's trials, and its count
        bool firstv = true;
        int cntv = 0;
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) {
            if (k < dl && av[k] == after) firstv = false;
            cntv += (av[k] == after);
        }
        // write-back of a bin the walker leaves in this step (all its visits),
        // by the shallowest on-path lane that ended in it
        {
            const bool own = onp && firstv && after != C;
            const bool entry_left = gl == G - 1 && C != ci && !b0_seen && hq > 0;
            if (LAZY) {
                // branch-free: lanes with nothing to write store to their own
                // slot of the mailbox (the bin index is clamped because a lane
                // off the true path may hold a bin outside the window)
                const int Xw = min(max(own ? after : ci, 0), T - 1);
                const int nq = (own ? cntv : 0) + (Xw == ci ? lq : tH[Xw]);
                int *dst = (own || entry_left) ? &tH[Xw] : &box->dummy[gl];
                *dst = nq;
            } else if (own || entry_left) {
                const int Xw = own ? after : ci;
                const bool isci = Xw == ci;
                const int cnt = own ? cntv : 0;
                const Val v0 = isci ? lbase : TB::load(tl, Xw);
                const int h0 = isci ? hbase : tH[Xw];
                const int nv = cnt + (isci ? lq : 0), nh = cnt + (isci ? hq : 0);
                const long long hv = (long long)(h0 < 0 ? 0 : h0) + nh;
                if (hv > 0x7FFFFFFFll) err = 1;
                tl[Xw] = TB::add(v0, nv, lnf, lnf32);
                tH[Xw] = (int32_t)hv;
            }
        }
        // the group adopts the state after the last trial
        e = ne;
        m = nm;
        {
            const bool same = C == ci;
            const int hC = tH[C];
            float bC;
            if constexpr (LAZY) {
                bC = scr32[C * SCR_STRIDE];
            } else {
                const Val lC = TB::load(tl, C);
                bC = TB::approx(lC);
                lbase = same ? lbase : lC;
            }
            hbase = same ? hbase : hC;
            base32 = same ? base32 : bC;
            lq = same ? lq + cC : cC + (LAZY ? hC : 0);
            hq = same ? hq + cC : cC;
            ci = C;
        }
        __syncwarp(gmask);
        u += (unsigned)(D + 1);
    }

    // ---- flush the current bin and the state
    if (gl == 0 && hq > 0) {
        if (LAZY) {
            tH[ci] = lq;
        } else {
            const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
            if (hv > 0x7FFFFFFFll) err = 1;
            tl[ci] = TB::add(lbase, lq, lnf, lnf32);
            tH[ci] = (int32_t)hv;
        }
    }
    __syncwarp(gmask);
    if (LAZY) {
        // fold the visits of this launch into the tables: bins not visited
        // keep their values and H (never visited: -1)
        for (int k = gl; k < T; k += G) {
            const int q = tH[k];
            if (q > 0) {
                const int h0 = gH[k];
                const long long hv = (long long)(h0 < 0 ? 0 : h0) + q;
                if (hv > 0x7FFFFFFFll) err = 1;
                g_tab[k] = TB::add(tl[k], q, lnf, lnf32);
                gH[k] = (int32_t)hv;
            }
        }
    } else if (SMT) {
        for (int k = gl; k < T; k += G) { g_tab[k] = tl[k]; gH[k] = tH[k]; }
    }
    if (REG) {
        for (int r = gl; r < L; r += G)
            p.spins[(size_t)r * p.nwalk + w] = (uint32_t)(lat64 >> (r * L)) & (uint32_t)((1ull << L) - 1);
    } else {
        for (int k = gl; k < nwords; k += G) p.spins[(size_t)k * p.nwalk + w] = lat[k];
    }
    if (gl == 0) {
        p.we[w] = e;
        p.wm[w] = m;
        p.wt[w] = t0 + u;
    }
    err = __any_sync(gmask, err);
    if (gl == 0 && err) atomicOr(&p.st->error, ERR_OVERFLOW);
}

// Shared memory per walker: ring, mailbox, lattice (16-byte padded) and, when staged,
// the tables (8-byte ln g entries in either format, 4-byte H, and for double
// tables a 4-byte float copy the screen reads).
size_t tree_smem_per_warp(const Params &p, bool smt)
{
    size_t b = RING * sizeof(RingEntry) + sizeof(Mailbox) + (((size_t)p.nwords * 4 + 15) & ~(size_t)15);
    if (smt) b += (size_t)p.T * (8 + sizeof(int32_t) + (p.precision == REWL_FP64 ? sizeof(float) : 0));
    return (b + 15) & ~(size_t)15;
}

// group: lanes per walker (8, 16 or 32); warps: warps per block.  One
// launch runs fewer than 2^31 trials per walker (launch_sweep splits).
cudaError_t launch_sweep_tree(const Params &p, uint64_t ntrials, int group, int warps, bool smt, cudaStream_t s)
{
    if (group != 8 && group != 16 && group != 32) group = 32;
    const size_t per = tree_smem_per_warp(p, smt);
    const int gpw = 32 / group;
    if (warps <= 0) warps = smt ? 1 : 4;
    // no more warps per block than the shared memory of one block holds
    const size_t max_smem = 227 * 1024;
    while (warps > 1 && per * (size_t)gpw * warps > max_smem) --warps;
    if (per * (size_t)gpw * warps > max_smem) return cudaErrorInvalidValue;
    const size_t smem = per * (size_t)gpw * warps;
    const int walkers_per_block = gpw * warps;
    const int blocks = (p.nwalk + walkers_per_block - 1) / walkers_per_block;
    const int threads = 32 * warps;
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, threads, smem, s>>>(p, (unsigned)ntrials, (int)per);
        return cudaGetLastError();
    };
#define REWL_TREE_G(W_, S_, P_)                                            \
    if (p.N <= 64 && W_ == 1) {                                            \
        if (group == 32) return go(k_sweep_tree<1, S_, 32, P_, true>);     \
        if (group == 16) return go(k_sweep_tree<1, S_, 16, P_, true>);     \
        return go(k_sweep_tree<1, S_, 8, P_, true>);                       \
    }                                                                      \
    if (group == 32) return go(k_sweep_tree<W_, S_, 32, P_, false>);       \
    if (group == 16) return go(k_sweep_tree<W_, S_, 16, P_, false>);       \
    return go(k_sweep_tree<W_, S_, 8, P_, false>);
#define REWL_TREE_P(W_, S_)                                                \
    if (p.precision == REWL_FP64) { REWL_TREE_G(W_, S_, REWL_FP64) }       \
    else if (p.precision == REWL_F32X2) { REWL_TREE_G(W_, S_, REWL_F32X2) } \
    else { REWL_TREE_G(W_, S_, REWL_F32) }
    if (p.wpr == 1) {
        if (smt) { REWL_TREE_P(1, true) } else { REWL_TREE_P(1, false) }
    } else {
        if (smt) { REWL_TREE_P(2, true) } else { REWL_TREE_P(2, false) }
    }
#undef REWL_TREE_P
#undef REWL_TREE_G
}

}  // namespace rewl

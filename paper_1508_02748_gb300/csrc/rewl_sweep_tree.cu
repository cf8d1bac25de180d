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
//   1. reads its trial's ring entry and the five spins around its site from
//      the committed lattice, corrected for the sites its history flips: the
//      ring entry carries, for each earlier trial of the step, which of the
//      five positions that trial's site is (a one-hot code made when the
//      ring was filled), so the correction is one mask and a fold;
//   2. takes the moves of the earlier trials of its history by shuffle from
//      the lanes that evaluated them and adds them up: its position (E, M)
//      and the positions after each earlier trial;
//   3. decides its own trial (Eq. 1) from the values the sequential chain
//      sees there, ln g(b) = base(b) + (H(b) + visits earlier in the step)
//      ln f.
// One ballot gives the true path from the root: a lane is on it iff the
// ballot bits of its ancestors are the outcomes its history assumes.  Lane k
// of the path knows how often its bin was visited on the path up to trial
// t+k (its own history's count plus one), so it writes that bin's H as the
// count it had plus those visits; the lanes write in path order (one store
// per depth, warp barriers between), so a bin visited again later ends with
// the larger count.  The leaf posts the final position, its visits on the
// path, its H and its screen value in a per-walker mailbox in shared memory
// (a register lattice also gets the path's flipped sites there), so the
// group adopts its new state without comparing the path's bins or reading
// the table again.
//
// Tables (exact formats only; REWL_F32 runs on the thread sampler): ln g(b)
// = base(b) + max(H(b), 0) ln f, the base fixed during an iteration, so a
// visit changes H alone and no floating-point table update runs here.  The
// decision is screened in float from a 32-bit screen per bin, S(b) =
// base(b) - c_w rounded to nearest (c_w one constant per walker, which
// cancels in the difference and keeps the screened magnitudes small), and
// re-taken exactly in double on near-ties.  Tables live in global memory
// (L1-cached) or, when small, are staged in shared memory for the launch
// (S and H; the bases are read only by the exact re-decision).
//
// The outcome is the sequential chain itself, trial for trial:
//   - random numbers are drawn per trial index from the TRIAL stream of
//     Philox4x32-10, independent of the state (a ring of 128 trials per
//     walker, refilled 64 at a time from the even trial at or below the
//     launch's first trial);
//   - base(b) + n ln f is evaluated exactly in double (fma; the compensated
//     pair converts exactly) and equals the sequential additions whenever
//     ln f = 2^-k and the values stay within 53 (pair: 48) bits;
//   - the float screen is decided only outside a margin that bounds its
//     error.  With S within 2^-24 |S| of base - c_w, the count converted to
//     float within 2^-24 of itself, one rounding in each fma and in the
//     difference, and the float ln u within 2^-22 (|ln u| + 1) of ln u (u
//     rounds with relative error below 2^-23, logf errs by at most one ulp),
//     the screened difference errs by less than
//         2^-21 (|c| + |n| + |S_c| + |S_n| + |ln u| + 1),
//     half of the margin M = 2^-20 (|c| + |n| + |S_c| + |S_n| + |ln u|) +
//     2^-20 used below.  Inside the margin the decision is re-taken from the
//     exact difference (out of line): against the float ln u where the two
//     are farther apart than 2^-20 (|ln u| + 1), else against ln u in double.
#include "rewl_tab.cuh"

namespace rewl {

using namespace tab;

namespace {

constexpr int RING = 128;   // trials buffered per walker

// One buffered trial (16 bytes, one shared-memory vector load).  Everything
// about a trial that does not depend on the walker's state is computed when
// the ring is refilled.
struct RingEntry {
    uint32_t a;    // five 6-bit fields at bits 0, 6, 12, 18, 24:
                   //   register lattice: bit indices i*L+j of the site and of its up,
                   //   down, left and right neighbours;
                   //   shared lattice: row i, column j, up row, down row, left column
    uint32_t b;    // bits 0-5: shared lattice: right column; bits 6-25: for lag
                   //   1..4 (5 bits each), which of (site, up, down, left, right)
                   //   is the site of trial t - lag (one-hot, or 0)
    uint32_t xu;   // acceptance word
    float lnu;     // ln u in float
};

// Per-walker exchange area of one step (shared memory, 16-byte aligned: it
// follows the ring).  The leaf's four words are written and read as one
// 16-byte vector.
struct Mailbox {
    int fsite[8];                  // register lattice: bit index flipped by trial t+k, 64 if none
    int leafC;                     // position e << 16 | m after the last trial
    int leafcC;                    // the path's visits of that bin
    int leafq;                     // its H as read this step (>= 0)
    float leafs;                   // its screen value
};
static_assert(offsetof(Mailbox, leafC) % 16 == 0 && (RING * sizeof(RingEntry)) % 16 == 0,
              "the leaf's post must be 16-byte aligned");

// Eq. 1 decided from the exact values (near-ties of the float screen only);
// kept out of line so none of it runs in the common case.  ccnt and ncnt
// are the visit counts the chain has at that point; the difference is exact
// in double.
template <class TB>
__device__ __noinline__ int exact_accept(const typename TB::Elem *gb, unsigned ci, int ccnt, unsigned ni, int ncnt,
                                         double lnf, uint32_t xu, float lnu32)
{
    const double delta = fma((double)ccnt, lnf, TB::exact(gb[ci])) - fma((double)ncnt, lnf, TB::exact(gb[ni]));
    if (delta >= 0.0) return 1;
    const double lu = (double)lnu32;
    const double band = (fabs(lu) + 1.0) * 0x1p-20;
    if (lu < delta - band) return 1;
    if (lu > delta + band) return 0;
    return log(unit_open_d(xu)) < delta ? 1 : 0;
}

template <int G>
struct TreeShape {
    static constexpr int DEPTH = G == 32 ? 4 : G == 16 ? 3 : G == 8 ? 2 : 1;
};

// Position code of a site for the relation codes: the bit index (register
// lattice) or row | column << 6 (shared lattice).
template <bool REG>
__device__ __forceinline__ uint32_t site_code(uint32_t a)
{
    return REG ? (a & 63u) : (a & 0xFFFu);
}

}  // namespace

// REG: the lattice (N <= 64 sites, bit i*L + j) is held in a 64-bit register
// by every lane; otherwise it lives in shared memory, one 32-bit word per row
// (two for L > 32).  SMT: S and H staged in shared memory for the launch.
template <int WPR, bool SMT, int G, int PREC, bool REG>
__global__ void __launch_bounds__(256) k_sweep_tree(Params p, unsigned ntrials, int smem_per_walker)
{
    using TB = Tab<PREC>;
    using Elem = typename TB::Elem;
    constexpr int DEPTH = TreeShape<G>::DEPTH;
    constexpr int GPW = 32 / G;   // walkers per warp
    constexpr unsigned GBITS = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
    constexpr unsigned RMASK = RING - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane & (G - 1), grp = lane / G;
    const unsigned gmask = GBITS << (grp * G);
    const int slot = wid * GPW + grp;   // walker slot within the block
    const int w = blockIdx.x * ((blockDim.x >> 5) * GPW) + slot;
    if (w >= p.nwalk || ntrials == 0) return;
    if (!p.active[w / p.W] || p.st->done) return;

    unsigned char *base = smem_raw + (size_t)slot * smem_per_walker;
    RingEntry *ring = reinterpret_cast<RingEntry *>(base);
    Mailbox *box = reinterpret_cast<Mailbox *>(base + RING * sizeof(RingEntry));
    uint32_t *lat = reinterpret_cast<uint32_t *>(base + RING * sizeof(RingEntry) + sizeof(Mailbox));
    const int L = p.L, nwords = L * WPR;
    const int T = p.T;
    const Elem *g_base = reinterpret_cast<const Elem *>(PREC == REWL_FP64 ? (const void *)p.lng : (const void *)p.lng2)
                       + (size_t)w * p.tstride;
    int32_t *gH = p.H + (size_t)w * p.tstride;
    const float *gS = p.scr + (size_t)w * p.tstride;
    const float *S;
    int32_t *Hh;
    if constexpr (SMT) {
        float *sS = reinterpret_cast<float *>(base + RING * sizeof(RingEntry) + sizeof(Mailbox) + ((nwords * 4 + 15) & ~15));
        int32_t *sH = reinterpret_cast<int32_t *>(sS + ((T + 3) & ~3));
        for (int k = gl; k < T; k += G) { sS[k] = gS[k]; sH[k] = gH[k]; }
        S = sS;
        Hh = sH;
    } else {
        S = gS;
        Hh = gH;
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
    const unsigned Tm1 = (unsigned)(T - 1);
    const double lnf = p.st->lnf;
    const float lnf32 = __double2float_rn(lnf);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t divL = p.divL;

    // this lane's node of the tree and the lanes holding its history's trials
    const int dl = 31 - __clz(gl + 1);
    const int hist = gl + 1 - (1 << dl);
    int srck[DEPTH];
    #pragma unroll
    for (int k = 0; k < DEPTH; ++k) srck[k] = grp * G + (1 << k) - 1 + (hist & ((1 << k) - 1));
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
    // relation fields of the lags whose trials the history accepts: trial
    // t+k (k < d) is lag d - k of this lane's trial
    uint32_t sel = 0;
    #pragma unroll
    for (int k = 0; k <= DEPTH; ++k)
        if (k < dl && ((hist >> k) & 1)) sel |= 0x1Fu << (5 * (dl - k - 1));

    // committed state (uniform over the group); positions are e << 16 | m
    int P0 = (p.we[w] << 16) | p.wm[w];
    int ci = ((P0 >> 16) - R.x) * wM + ((P0 & 0xFFFF) - R.z);
    int lq = max(Hh[ci], 0);        // H of the current bin, visits of this step excluded
    int hq = 0;                     // visits of the current bin not yet written to H
    float base32 = S[ci];
    const unsigned long long t0 = p.wt[w];
    const unsigned r0 = (unsigned)t0 & RMASK;
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
                        en.a = i | (j << 6) | (iu << 12) | (id << 18) | (jl << 24);
                        en.b = jr;
                    }
                    en.xu = xu;
                    en.lnu = logf(__fmaf_rn(__uint2float_rn(xu), 0x1p-32f, 0x1p-33f));
                    ring[(unsigned)(2 * c + hh) & RMASK] = en;
                }
            }
            __syncwarp(gmask);
            // relation codes of the 64 new trials to the DEPTH trials before each
            #pragma unroll
            for (int r = 0; r < 64 / G; ++r) {
                const unsigned q = (unsigned)(2 * (c0 + cfill)) + (unsigned)(gl + r * G);
                const uint32_t a = ring[q & RMASK].a, b = ring[q & RMASK].b;
                uint32_t pos[5];
                if (REG) {
                    #pragma unroll
                    for (int f = 0; f < 5; ++f) pos[f] = (a >> (6 * f)) & 63u;
                } else {
                    const uint32_t row = a & 63u, colbits = a & (63u << 6);
                    pos[0] = a & 0xFFFu;
                    pos[1] = ((a >> 12) & 63u) | colbits;
                    pos[2] = ((a >> 18) & 63u) | colbits;
                    pos[3] = row | (((a >> 24) & 63u) << 6);
                    pos[4] = row | ((b & 63u) << 6);
                }
                uint32_t rel = 0;
                #pragma unroll
                for (int lag = 1; lag <= DEPTH; ++lag) {
                    const uint32_t f = site_code<REG>(ring[(q - lag) & RMASK].a);
                    uint32_t oh = 0;
                    #pragma unroll
                    for (int k = 0; k < 5; ++k) oh |= (uint32_t)(f == pos[k]) << k;
                    rel |= oh << (5 * (lag - 1));
                }
                ring[q & RMASK].b = b | (rel << 6);
            }
            cfill += 32;
            ufill = 2 * cfill - (unsigned)(t0 & 1ull);
            __syncwarp(gmask);
        }
        const unsigned left = ntrials - u;
        const int D = left > (unsigned)DEPTH ? DEPTH : (int)left - 1;
        const unsigned rb = r0 + u;

        // ---- 1. own trial under own history: the five spins
        const RingEntry me = ring[(rb + dl) & RMASK];
        uint32_t v5;
        if (REG) {
            v5 = ((uint32_t)(lat64 >> (me.a & 63u)) & 1u)
               | (((uint32_t)(lat64 >> ((me.a >> 6) & 63u)) & 1u) << 1)
               | (((uint32_t)(lat64 >> ((me.a >> 12) & 63u)) & 1u) << 2)
               | (((uint32_t)(lat64 >> ((me.a >> 18) & 63u)) & 1u) << 3)
               | (((uint32_t)(lat64 >> ((me.a >> 24) & 63u)) & 1u) << 4);
        } else {
            const uint32_t i = me.a & 63u, j = (me.a >> 6) & 63u, iu = (me.a >> 12) & 63u, id = (me.a >> 18) & 63u;
            const uint32_t jl = (me.a >> 24) & 63u, jr = me.b & 63u;
            const uint32_t qj = (WPR == 1) ? 0 : (j >> 5);
            const uint32_t wc = lat[i * WPR + qj], wu = lat[iu * WPR + qj], wd = lat[id * WPR + qj];
            const uint32_t wl = (WPR == 1) ? wc : lat[i * WPR + (jl >> 5)];
            const uint32_t wr = (WPR == 1) ? wc : lat[i * WPR + (jr >> 5)];
            v5 = ((wc >> (j & 31)) & 1u) | (((wu >> (j & 31)) & 1u) << 1) | (((wd >> (j & 31)) & 1u) << 2)
               | (((wl >> (jl & 31)) & 1u) << 3) | (((wr >> (jr & 31)) & 1u) << 4);
        }
        {
            const uint32_t corr = (me.b >> 6) & sel;
            v5 ^= (corr ^ (corr >> 5) ^ (corr >> 10) ^ (corr >> 15)) & 0x1Fu;
        }
        const int sup = (int)(v5 & 1u);
        const int nup = __popc(v5 & 0x1Eu);
        const int de_own = sup ? nup - 2 : 2 - nup;
        const int dm_own = sup ? -1 : 1;
        const int pk = de_own * 65536 + dm_own;   // move as a position difference

        // ---- 2. the history's earlier trials: the move of trial k under the
        // history's first k outcomes is the own move of lane 2^k - 1 + (h mod 2^k);
        // a history that accepts a move out of the window is never the true path
        int Pc = P0;
        int vb[DEPTH];               // position after each earlier trial (-1 past the own depth)
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            const int x = __shfl_sync(gmask, pk, srck[k]);
            if ((hist >> k) & 1) Pc += x;
            vb[k] = k < dl ? Pc : -1;
        }
        const int Pn = Pc + pk;
        const int ce = Pc >> 16, cm = Pc & 0xFFFF;
        const int cidx = (ce - R.x) * wM + (cm - R.z);
        const int nidx = cidx + de_own * wM + dm_own;
        const bool live = dl <= D && (unsigned)(ce + de_own - R.x) <= spanE && (unsigned)(cm + dm_own - R.z) <= spanM;

        // ---- 3. decision of the own trial (Eq. 1); off-path lanes may hold
        // positions outside the window, so their reads are clamped
        const unsigned cu = min((unsigned)cidx, Tm1), nu = min((unsigned)nidx, Tm1);
        // a lane whose bin is the walker's committed bin takes S and H from
        // registers (base32, lq); with the tables in global memory it also
        // skips their load (in shared memory the predicate costs more than the load)
        const bool c0p = !SMT && Pc == P0, n0p = !SMT && Pn == P0;
        const float cs_m = c0p ? 0.f : S[cu], ns_m = n0p ? 0.f : S[nu];
        const int hc = c0p ? 0 : max(Hh[cu], 0), hn = n0p ? 0 : max(Hh[nu], 0);
        int vcur = 0, vnew = 0;
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            vcur += (vb[k] == Pc);
            vnew += (vb[k] == Pn);
        }
        const bool c0b = Pc == P0, n0b = Pn == P0;
        const float cs = c0b ? base32 : cs_m, ns = n0b ? base32 : ns_m;
        const int ccnt = vcur + (c0b ? lq : hc), ncnt = vnew + (n0b ? lq : hn);
        const float c32 = __fmaf_rn(__int2float_rn(ccnt), lnf32, cs);
        const float n32 = __fmaf_rn(__int2float_rn(ncnt), lnf32, ns);
        const float d32 = __fsub_rn(c32, n32);
        // the terms known before c and n are summed first (shorter chain; the
        // margin's factor-two slack over the error bound covers either order)
        const float M = __fmaf_rn((fabsf(c32) + fabsf(n32)) + (fabsf(cs) + fabsf(ns) + fabsf(me.lnu)), 0x1p-20f,
                                  0x1p-20f);
        int acc = (me.lnu < d32 - M) ? 1 : 0;
        if (live && !acc && !(me.lnu > d32 + M))
            acc = exact_accept<TB>(g_base, cu, ccnt, nu, ncnt, lnf, me.xu, me.lnu);
        acc = live ? acc : 0;
        const int after = acc ? Pn : Pc;          // position after the own trial, under the own history

        // ---- the true path: the lanes whose ancestors decided as their history assumes
        const unsigned bal = (__ballot_sync(gmask, acc) >> (grp * G)) & GBITS;
        const bool onp = dl <= D && ((bal ^ want) & anc) == 0u;

        // ---- commit: the on-path lane of depth k takes trial t+k.  Its bin has
        // cupto path visits up to and including this trial, so its H becomes
        // cupto plus the H it had (the current bin: lq).
        const int aq = acc ? hn : hc;             // H of `after` as read (unless it is the current bin)
        const int cupto = (acc ? vnew : vcur) + 1;
        const int val = cupto + (after == P0 ? lq : aq);
        const unsigned aidx = acc ? nu : cu;
        if (onp) {
            if (REG) box->fsite[dl] = acc ? (int)(me.a & 63u) : 64;
            if (dl == D)      // one 16-byte store: position, visits, H, screen
                *reinterpret_cast<int4 *>(&box->leafC) = make_int4(after, cupto, aq, __float_as_int(acc ? ns : cs));
            err |= val < 0;
        }
        // H of the bins visited in this step, in path order: the pending count of
        // the start bin, then each trial's bin with its visits so far; a bin
        // visited again later in the step is overwritten with the larger count,
        // so every bin ends with all its visits (the warp barriers order the
        // stores of different lanes to one address)
        if (gl == 0 && hq > 0) Hh[ci] = lq;
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) {
            __syncwarp(gmask);
            if (onp && dl == k) Hh[aidx] = val;
        }
        __syncwarp(gmask);
        const int4 lb = *reinterpret_cast<const int4 *>(&box->leafC);   // the leaf's post
        const int C = lb.x, cC = lb.y;
        if (REG) {
            #pragma unroll
            for (int k = 0; k <= DEPTH; ++k) {
                if (k <= D) {
                    const int f = box->fsite[k];
                    lat64 ^= (unsigned long long)(f < 64) << (f & 63);
                }
            }
        } else if (onp && acc) {
            const uint32_t fi = me.a & 63u, fj = (me.a >> 6) & 63u;
            atomicXor(&lat[fi * WPR + ((WPR == 1) ? 0 : (fj >> 5))], 1u << (fj & 31));
        }
        // the group adopts the state after the last trial
        {
            const bool same = C == P0;
            const int nlq = (same ? lq : lb.z) + cC;
            const float ns32 = __int_as_float(lb.w);
            hq = same ? hq + cC : cC;
            lq = nlq;
            err |= nlq < 0;
            if (!same) {
                base32 = ns32;
                ci = ((C >> 16) - R.x) * wM + ((C & 0xFFFF) - R.z);
            }
            P0 = C;
        }
        __syncwarp(gmask);
        u += (unsigned)(D + 1);
    }

    // ---- flush the current bin and the state
    if (gl == 0 && hq > 0) Hh[ci] = lq;
    __syncwarp(gmask);
    if constexpr (SMT) {
        for (int k = gl; k < T; k += G) gH[k] = Hh[k];
    }
    if (REG) {
        for (int r = gl; r < L; r += G)
            p.spins[(size_t)r * p.nwalk + w] = (uint32_t)(lat64 >> (r * L)) & (uint32_t)((1ull << L) - 1);
    } else {
        for (int k = gl; k < nwords; k += G) p.spins[(size_t)k * p.nwalk + w] = lat[k];
    }
    if (gl == 0) {
        p.we[w] = P0 >> 16;
        p.wm[w] = P0 & 0xFFFF;
        p.wt[w] = t0 + u;
    }
    err = __any_sync(gmask, err);
    if (gl == 0 && err) atomicOr(&p.st->error, ERR_OVERFLOW);
}

// Shared memory per walker: ring, mailbox, lattice (16-byte padded) and, when
// staged, S (4 bytes per bin, padded to 16 bytes) and H (4 bytes per bin).
size_t tree_smem_per_warp(const Params &p, bool smt)
{
    size_t b = RING * sizeof(RingEntry) + sizeof(Mailbox) + (((size_t)p.nwords * 4 + 15) & ~(size_t)15);
    if (smt) b += (((size_t)p.T + 3) & ~(size_t)3) * 4 + (size_t)p.T * 4;
    return (b + 15) & ~(size_t)15;
}

// group: lanes per walker (8, 16 or 32); warps: warps per block.  One
// launch runs fewer than 2^31 trials per walker (launch_sweep splits).
// Exact table formats only.
cudaError_t launch_sweep_tree(const Params &p, uint64_t ntrials, int group, int warps, bool smt, cudaStream_t s)
{
    if (p.precision != REWL_FP64 && p.precision != REWL_F32X2) return cudaErrorInvalidValue;
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
    if (p.lattice_reg && W_ == 1) {                                        \
        if (group == 32) return go(k_sweep_tree<1, S_, 32, P_, true>);     \
        if (group == 16) return go(k_sweep_tree<1, S_, 16, P_, true>);     \
        return go(k_sweep_tree<1, S_, 8, P_, true>);                       \
    }                                                                      \
    if (group == 32) return go(k_sweep_tree<W_, S_, 32, P_, false>);       \
    if (group == 16) return go(k_sweep_tree<W_, S_, 16, P_, false>);       \
    return go(k_sweep_tree<W_, S_, 8, P_, false>);
#define REWL_TREE_P(W_, S_)                                                \
    if (p.precision == REWL_FP64) { REWL_TREE_G(W_, S_, REWL_FP64) }       \
    else { REWL_TREE_G(W_, S_, REWL_F32X2) }
    if (p.wpr == 1) {
        if (smt) { REWL_TREE_P(1, true) } else { REWL_TREE_P(1, false) }
    } else {
        if (smt) { REWL_TREE_P(2, true) } else { REWL_TREE_P(2, false) }
    }
#undef REWL_TREE_P
#undef REWL_TREE_G
}

}  // namespace rewl

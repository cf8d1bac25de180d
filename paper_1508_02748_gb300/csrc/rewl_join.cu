// Final merge, join and normalisation of librewl, all in FP64 on the device
// (arXiv:1508.02748, Sec. 2, Eqs. 3-4):
//   1. each window's walkers are merged: every walker is shifted by the mean,
//      over the bins all walkers of the window visited, of its difference to
//      walker 0; each bin is the mean over the walkers that visited it;
//   2. within each row of windows (same M range), pieces are joined along E:
//      g(E) = sum_M g(E,M) (Eq. 3) of each piece, beta(E) = d ln g / dE as the
//      forward difference over one bin (dE = 4), E_mat = the overlap bin with
//      minimal |beta_i - beta_j| (lowest on ties, never below the previous
//      matching point), piece j rescaled to agree with piece i at E_mat, and
//      piece i used for E < E_mat, piece j for E >= E_mat (Eq. 4);
//   3. the rows are joined along M by the same rule on g(M) = sum_E g(E,M)
//      (dM = 2), "one at a time" as Sec. 2 prescribes for both axes split;
//   4. the joined table is shifted so that sum g = 2^N.
// Loops that the sums depend on run in a fixed order (one thread per output
// element), so results differ from a serial evaluation only by the rounding
// of exp/log and of the final parallel normalisation sum.
#include <math.h>

#include <algorithm>

#include <math_constants.h>

#include "rewl_internal.cuh"

namespace rewl {

namespace {

// ln g of table entry i: base + max(H, 0) ln f in the exact formats (a
// caller's plain table is read with ln f = 0), the stored value for REWL_F32.
__device__ __forceinline__ double lng_at(const Params &p, size_t i)
{
    if (p.precision == REWL_F32) return (double)p.lng1[i];
    double b;
    if (p.precision == REWL_FP64) {
        b = p.lng[i];
    } else {
        const float2 v = p.lng2[i];
        b = (double)v.x + (double)v.y;
    }
    return fma((double)max(p.H[i], 0), p.st->lnf, b);
}

__device__ __forceinline__ bool all_seen(const Params &p, int win, int bin)
{
    for (int k = 0; k < p.W; ++k)
        if (k != p.join_exclude && p.H[(size_t)(win * p.W + k) * p.tstride + bin] < 0) return false;
    return true;
}

// Serial log-sum-exp in index order: max, then sum of exp(v - max) over the
// finite entries.
template <typename F>
__device__ double lse_serial(int n, F get)
{
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i) mx = fmax(mx, get(i));
    if (mx == -INFINITY) return -INFINITY;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        const double v = get(i);
        if (v != -INFINITY) acc += exp(v - mx);
    }
    return mx + log(acc);
}

// Matching point (Eq. 4) between marginals Ga, Gb over [lo, hi], q >= floor:
// the overlap bin q minimising |beta_a(q) - beta_b(q)|, beta the forward
// difference over one bin divided by the bin step, taken only where both
// marginals are finite at q and q + 1; the lowest such q on ties.  Without
// any, the lowest q where both are finite; -1 if none.
// It is computed by a whole block (every thread calls it and gets the
// result): each thread scans a stride of q keeping its first minimum, and
// the (difference, q) pairs are reduced lexicographically, so the lowest q
// wins ties.
constexpr int MATCH_THREADS = 256;

__device__ void block_min_pair(double &d, int &q, double *s_d, int *s_q)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xFFFFFFFFu, d, o);
        const int oq = __shfl_xor_sync(0xFFFFFFFFu, q, o);
        if (od < d || (od == d && oq < q)) { d = od; q = oq; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { s_d[threadIdx.x >> 5] = d; s_q[threadIdx.x >> 5] = q; }
    __syncthreads();
    d = s_d[0];
    q = s_q[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
        if (s_d[k] < d || (s_d[k] == d && s_q[k] < q)) { d = s_d[k]; q = s_q[k]; }
}

__device__ int match_point_block(const double *Ga, const double *Gb, int lo, int hi, int floor_p, double step)
{
    __shared__ double s_d[MATCH_THREADS / 32];
    __shared__ int s_q[MATCH_THREADS / 32];
    const int start = lo > floor_p ? lo : floor_p;
    double bestd = INFINITY;
    int best = 0x7FFFFFFF;
    for (int q = start + (int)threadIdx.x; q + 1 <= hi; q += blockDim.x) {
        if (Ga[q] == -INFINITY || Ga[q + 1] == -INFINITY) continue;
        if (Gb[q] == -INFINITY || Gb[q + 1] == -INFINITY) continue;
        const double ba = (Ga[q + 1] - Ga[q]) / step;
        const double bb = (Gb[q + 1] - Gb[q]) / step;
        const double d = fabs(ba - bb);
        if (d < bestd) { bestd = d; best = q; }
    }
    block_min_pair(bestd, best, s_d, s_q);
    if (best != 0x7FFFFFFF) return best;
    double z = 0.0;
    best = 0x7FFFFFFF;
    for (int q = start + (int)threadIdx.x; q <= hi; q += blockDim.x)
        if (Ga[q] != -INFINITY && Gb[q] != -INFINITY) { best = q; break; }
    block_min_pair(z, best, s_d, s_q);
    return best == 0x7FFFFFFF ? -1 : best;
}

}  // namespace

// 1a. Offsets: one block per (window, walker), relative to the first walker
// taking part (walker join_exclude, if >= 0, is left out: the jackknife
// replicates).  The block's threads take the bins in strides and reduce
// their sums in a fixed order.
constexpr int MERGE_OFF_THREADS = 256;

__global__ void __launch_bounds__(MERGE_OFF_THREADS) k_merge_off(Params p, JoinScratch j)
{
    const int idx = blockIdx.x;
    if (idx >= p.nwalk) return;
    const int win = idx / p.W, k = idx % p.W;
    if (!p.active[win]) return;
    const int ref = p.join_exclude == 0 ? 1 : 0;   // the first walker taking part
    if (k == ref || k == p.join_exclude) {
        if (threadIdx.x == 0) j.off[idx] = 0.0;
        return;
    }
    const size_t b0 = (size_t)(win * p.W + ref) * p.tstride, bk = (size_t)idx * p.tstride;
    double acc = 0.0;
    long long common = 0;
    for (int i = threadIdx.x; i < p.T; i += MERGE_OFF_THREADS) {
        if (!all_seen(p, win, i)) continue;
        acc += lng_at(p, bk + i) - lng_at(p, b0 + i);
        ++common;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        common += __shfl_down_sync(0xFFFFFFFFu, common, o);
    }
    __shared__ double s_acc[MERGE_OFF_THREADS / 32];
    __shared__ long long s_cnt[MERGE_OFF_THREADS / 32];
    if ((threadIdx.x & 31) == 0) { s_acc[threadIdx.x >> 5] = acc; s_cnt[threadIdx.x >> 5] = common; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    acc = 0.0;
    common = 0;
    for (int w = 0; w < MERGE_OFF_THREADS / 32; ++w) { acc += s_acc[w]; common += s_cnt[w]; }
    if (common == 0) { atomicExch(&p.st->join_error, 1); j.off[idx] = 0.0; return; }
    j.off[idx] = acc / (double)common;
}

// 1b. Merged piece: one thread per (window, bin), walkers in order.
__global__ void k_merge(Params p, JoinScratch j)
{
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)p.nwin * p.T) return;
    const int win = (int)(idx / p.T), bin = (int)(idx % p.T);
    double *out = j.piece + (size_t)win * p.tstride + bin;
    if (!p.active[win]) { *out = -INFINITY; return; }
    double acc = 0.0;
    int cnt = 0;
    for (int k = 0; k < p.W; ++k) {
        const size_t q = (size_t)(win * p.W + k) * p.tstride + bin;
        if (k == p.join_exclude || p.H[q] < 0) continue;
        acc += lng_at(p, q) - j.off[win * p.W + k];
        ++cnt;
    }
    *out = cnt ? acc / (double)cnt : -INFINITY;
}

// 2a. E marginal of each piece over its M range (Eq. 3).
__global__ void k_marg_piece(Params p, JoinScratch j)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p.nwin * p.wE) return;
    const int win = idx / p.wE, el = idx % p.wE;
    const double *row = j.piece + (size_t)win * p.tstride + (size_t)el * p.wM;
    j.GE[idx] = p.active[win] ? lse_serial(p.wM, [&](int i) { return row[i]; }) : -INFINITY;
}

// 2b. One block per row b: chain of E matching points along the row (the
// chain is sequential; each matching point and slice rule is block-parallel).
__global__ void __launch_bounds__(MATCH_THREADS) k_match_e(Params p, JoinScratch j, double *gbuf)
{
    const int b = blockIdx.x;
    if (b >= p.nM) return;
    const int nE = p.nE, B = p.N + 1, t0 = threadIdx.x == 0;
    double *Ga = gbuf + (size_t)b * 2 * B, *Gb = Ga + B;
    __shared__ int s_first, s_last, s_bad;
    if (t0) {
        for (int a = 0; a < nE; ++a) {
            j.efrom[b * nE + a] = 0; j.eto[b * nE + a] = 0; j.eshift[b * nE + a] = 0.0;
            if (a < nE - 1) j.ematch[b * (nE - 1) + a] = -1;
        }
        if (nE == 1) j.ematch[b] = -1;
        int first = -1, last = -1, bad = 0;
        for (int a = 0; a < nE; ++a)
            if (p.active[b * nE + a]) { if (first < 0) first = a; last = a; }
        j.rowok[b] = first >= 0;
        for (int a = first; first >= 0 && a <= last; ++a)
            if (!p.active[b * nE + a]) bad = 1;
        if (bad) atomicExch(&p.st->join_error, 2);
        s_first = first; s_last = last; s_bad = bad;
    }
    __syncthreads();
    const int first = s_first, last = s_last;
    if (first < 0 || s_bad) return;
    double shift = 0.0;
    if (p.join_rule == 1)
        for (int ml = threadIdx.x; ml < p.wM; ml += blockDim.x) j.eslice[(size_t)(b * nE + first) * p.wM + ml] = 0.0;
    int from = p.rect[b * nE + first].x;
    for (int a = first; a <= last; ++a) {
        const int A = b * nE + a;
        const int4 RA = p.rect[A];
        int to;
        double next_shift = 0.0;
        __syncthreads();                      // the last piece's buffers and slices are complete
        if (a < last) {
            const int4 RB = p.rect[A + 1];
            for (int e = threadIdx.x; e < B; e += blockDim.x) {
                Ga[e] = (e >= RA.x && e <= RA.y) ? j.GE[A * p.wE + (e - RA.x)] : -INFINITY;
                Gb[e] = (e >= RB.x && e <= RB.y) ? j.GE[(A + 1) * p.wE + (e - RB.x)] : -INFINITY;
            }
            __syncthreads();
            const int q = match_point_block(Ga, Gb, RB.x, RA.y, from, 4.0);
            if (q < 0) { if (t0) atomicExch(&p.st->join_error, 3); return; }
            if (t0) j.ematch[b * (nE - 1) + a] = q;
            next_shift = shift + (Ga[q] - Gb[q]);
            if (p.join_rule == 1) {
                // the next piece's M slices: each matched at (E_mat, M) where
                // both pieces have the bin, else by the marginals
                const double *pa = j.piece + (size_t)A * p.tstride + (size_t)(q - RA.x) * p.wM;
                const double *pb = j.piece + (size_t)(A + 1) * p.tstride + (size_t)(q - RB.x) * p.wM;
                const double *sa = j.eslice + (size_t)A * p.wM;
                double *sb = j.eslice + (size_t)(A + 1) * p.wM;
                for (int ml = threadIdx.x; ml < p.wM; ml += blockDim.x) {
                    const double va = pa[ml], vb = pb[ml];
                    sb[ml] = sa[ml] + ((va != -INFINITY && vb != -INFINITY) ? va - vb : Ga[q] - Gb[q]);
                }
            }
            to = q;
        } else {
            to = RA.y + 1;
        }
        if (t0) { j.efrom[A] = from; j.eto[A] = to; j.eshift[A] = shift; }
        shift = next_shift;
        from = to;
    }
}

// Value of row b at (e, m): the piece covering e in that row, shifted.
__device__ __forceinline__ double row_value(const Params &p, const JoinScratch &j, int b, int e, int m)
{
    for (int a = 0; a < p.nE; ++a) {
        const int A = b * p.nE + a;
        if (e >= j.efrom[A] && e < j.eto[A]) {
            const int4 R = p.rect[A];
            if (m < R.z || m > R.w) return -INFINITY;
            const double v = j.piece[(size_t)A * p.tstride + (size_t)(e - R.x) * p.wM + (m - R.z)];
            const double c = p.join_rule == 1 ? j.eslice[(size_t)A * p.wM + (m - R.z)] : j.eshift[A];
            return v == -INFINITY ? v : v + c;
        }
    }
    return -INFINITY;
}

// 3a. M marginal of each row: F_b(m) = ln sum_E g_b(E, m), e ascending.
__global__ void k_marg_row(Params p, JoinScratch j)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int B = p.N + 1;
    if (idx >= p.nM * B) return;
    const int b = idx / B, m = idx % B;
    if (!j.rowok[b]) { j.F[idx] = -INFINITY; return; }
    j.F[idx] = lse_serial(B, [&](int e) { return row_value(p, j, b, e, m); });
}

// 3b. One block: chain of M matching points over the rows (sequential
// chain, block-parallel matching point and slice rule).
__global__ void __launch_bounds__(MATCH_THREADS) k_match_m(Params p, JoinScratch j)
{
    const int nM = p.nM, nE = p.nE, B = p.N + 1, t0 = threadIdx.x == 0;
    __shared__ int s_first, s_last, s_bad;
    if (t0) {
        for (int b = 0; b < nM; ++b) { j.mfrom[b] = 0; j.mto[b] = 0; j.mshift[b] = 0.0; }
        for (int b = 0; b < (nM > 1 ? nM - 1 : 1); ++b) j.mmatch[b] = -1;
        int first = -1, last = -1, bad = 0;
        for (int b = 0; b < nM; ++b) if (j.rowok[b]) { if (first < 0) first = b; last = b; }
        if (first < 0) { bad = 1; atomicExch(&p.st->join_error, 4); }
        for (int b = first; first >= 0 && b <= last; ++b) if (!j.rowok[b]) bad = 1;
        if (bad && first >= 0) atomicExch(&p.st->join_error, 5);
        s_first = first; s_last = last; s_bad = bad;
    }
    __syncthreads();
    const int first = s_first, last = s_last;
    if (s_bad) return;
    double shift = 0.0;
    if (p.join_rule == 1)
        for (int e = threadIdx.x; e < B; e += blockDim.x) j.mslice[(size_t)first * B + e] = 0.0;
    int from = p.rect[first * nE].z;
    for (int b = first; b <= last; ++b) {
        int to;
        double next_shift = 0.0;
        __syncthreads();                      // the last row's slices are complete
        if (b < last) {
            const double *Ga = j.F + (size_t)b * B, *Gb = j.F + (size_t)(b + 1) * B;
            const int lo = p.rect[(b + 1) * nE].z, hi = p.rect[b * nE].w;
            const int q = match_point_block(Ga, Gb, lo, hi, from, 2.0);
            if (q < 0) { if (t0) atomicExch(&p.st->join_error, 6); return; }
            if (t0) j.mmatch[b] = q;
            next_shift = shift + (Ga[q] - Gb[q]);
            if (p.join_rule == 1)
                for (int e = threadIdx.x; e < B; e += blockDim.x) {
                    const double va = row_value(p, j, b, e, q), vb = row_value(p, j, b + 1, e, q);
                    j.mslice[(size_t)(b + 1) * B + e] = j.mslice[(size_t)b * B + e]
                        + ((va != -INFINITY && vb != -INFINITY) ? va - vb : Ga[q] - Gb[q]);
                }
            to = q;
        } else {
            to = p.rect[b * nE].w + 1;
        }
        if (t0) { j.mfrom[b] = from; j.mto[b] = to; j.mshift[b] = shift; }
        shift = next_shift;
        from = to;
    }
}

// 3c. Assemble the joined table.
__global__ void k_assemble(Params p, JoinScratch j)
{
    const int B = p.N + 1;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * B) return;
    const int e = (int)(idx / B), m = (int)(idx % B);
    double v = -INFINITY;
    for (int b = 0; b < p.nM; ++b) {
        if (m >= j.mfrom[b] && m < j.mto[b]) {
            const double r = row_value(p, j, b, e, m);
            const double c = p.join_rule == 1 ? j.mslice[(size_t)b * B + e] : j.mshift[b];
            v = r == -INFINITY ? r : r + c;
            break;
        }
    }
    j.J[idx] = v;
}

// 4. Normalisation: max, then sum of exp(v - max), block partials in red[].
__global__ void k_red_max(const double *v, size_t n, double *red)
{
    double mx = -INFINITY;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mx = fmax(mx, v[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, s[k]);
        red[blockIdx.x] = mx;
    }
}

// Block partials red[0..nblk) folded once, by one block: red[RED_MAX] = the max.
constexpr int RED_MAX = 1024, RED_SHIFT = 1025;

__global__ void k_red_fold_max(double *red, int nblk)
{
    double mx = -INFINITY;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) mx = fmax(mx, red[k]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, s[k]);
        red[RED_MAX] = mx;
    }
}

__global__ void k_red_sumexp(const double *v, size_t n, double *red)
{
    const double mx = red[RED_MAX];
    double acc = 0.0;
    if (mx != -INFINITY)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
            if (v[i] != -INFINITY) acc += exp(v[i] - mx);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) acc += s[k];
        red[512 + blockIdx.x] = acc;
    }
}

// Sum partials red[512..512+nblk) folded in a fixed order; red[RED_SHIFT] =
// N ln 2 - ln sum g, the shift that makes sum g = 2^N.
__global__ void k_red_fold_sum(double *red, int nblk, int N)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += red[512 + k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) acc += s[k];
        red[RED_SHIFT] = (double)N * log(2.0) - (red[RED_MAX] + log(acc));
    }
}

__global__ void k_normalise(double *v, size_t n, const double *red)
{
    const double c = red[RED_SHIFT];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (v[i] != -INFINITY) v[i] += c;
}

cudaError_t launch_join(const Params &p, const JoinScratch &j, cudaStream_t s)
{
    const int B = p.N + 1;
    k_merge_off<<<p.nwalk, MERGE_OFF_THREADS, 0, s>>>(p, j);
    const size_t nb = (size_t)p.nwin * p.T;
    k_merge<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(p, j);
    k_marg_piece<<<(p.nwin * p.wE + 127) / 128, 128, 0, s>>>(p, j);
    k_match_e<<<p.nM, MATCH_THREADS, 0, s>>>(p, j, j.gbuf);
    k_marg_row<<<(p.nM * B + 127) / 128, 128, 0, s>>>(p, j);
    k_match_m<<<1, MATCH_THREADS, 0, s>>>(p, j);
    const size_t nJ = (size_t)B * B;
    k_assemble<<<(unsigned)((nJ + 255) / 256), 256, 0, s>>>(p, j);
    // normalisation: block maxima, one fold, block sums of exp(v - max), one
    // fold into the shift, shift applied (grids sized to the table, <= 512)
    const int nblk = (int)std::min<size_t>(512, (nJ + 255) / 256);
    k_red_max<<<nblk, 256, 0, s>>>(j.J, nJ, j.red);
    k_red_fold_max<<<1, 512, 0, s>>>(j.red, nblk);
    k_red_sumexp<<<nblk, 256, 0, s>>>(j.J, nJ, j.red);
    k_red_fold_sum<<<1, 512, 0, s>>>(j.red, nblk, p.N);
    k_normalise<<<nblk, 256, 0, s>>>(j.J, nJ, j.red);
    return cudaGetLastError();
}

// Eq. 3 on the joined table: ln sum_m g(e, m), m ascending.
__global__ void k_marg_out(Params p, JoinScratch j)
{
    const int B = p.N + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B) return;
    const double *row = j.J + (size_t)e * B;
    j.marg[e] = lse_serial(B, [&](int i) { return row[i]; });
}

cudaError_t launch_marginal_e(const Params &p, const JoinScratch &j, cudaStream_t s)
{
    k_marg_out<<<(p.N + 1 + 127) / 128, 128, 0, s>>>(p, j);
    return cudaGetLastError();
}

// Jackknife accumulation over replicates k = 0..W-1 (walker k left out of
// every window's merge): differences to replicate 0 are summed; an entry that
// is missing (-inf) in any replicate is marked NaN in jk_ref.
__global__ void k_jk_accum(JoinScratch j, const double *x, size_t n, int k)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        if (k == 0) {
            j.jk_ref[i] = isfinite(v) ? v : NAN;
            j.jk_sum[i] = 0.0;
            j.jk_sq[i] = 0.0;
        } else if (!isfinite(v)) {
            j.jk_ref[i] = NAN;
        } else {
            const double d = v - j.jk_ref[i];
            j.jk_sum[i] += d;
            j.jk_sq[i] += d * d;
        }
    }
}

__global__ void k_jk_final(JoinScratch j, double *mean, double *err, size_t n, int W)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double r = j.jk_ref[i];
        if (isnan(r)) {
            mean[i] = -INFINITY;
            err[i] = NAN;
            continue;
        }
        const double s1 = j.jk_sum[i], s2 = j.jk_sq[i];
        mean[i] = r + s1 / W;
        const double var = (double)(W - 1) / W * (s2 - s1 * s1 / W);
        err[i] = sqrt(var > 0.0 ? var : 0.0);
    }
}

cudaError_t launch_jk_accum(const JoinScratch &j, const double *x, size_t n, int k, cudaStream_t s)
{
    k_jk_accum<<<256, 256, 0, s>>>(j, x, n, k);
    return cudaGetLastError();
}

cudaError_t launch_jk_final(const JoinScratch &j, double *mean, double *err, size_t n, int W, cudaStream_t s)
{
    k_jk_final<<<256, 256, 0, s>>>(j, mean, err, n, W);
    return cudaGetLastError();
}

// Eq. 5 per bin: |g_a - g_b| / ((g_a + g_b) / 2) = 2 tanh(|ln g_a - ln g_b| / 2),
// 2 where one table is empty, NaN where both are.
__global__ void k_rel_diff(const double *a, const double *b, double *out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = a[i], y = b[i];
        const bool ex = x == -CUDART_INF, ey = y == -CUDART_INF;
        out[i] = (ex && ey) ? CUDART_NAN : (ex || ey) ? 2.0 : 2.0 * tanh(0.5 * fabs(x - y));
    }
}

cudaError_t launch_rel_diff(const double *a, const double *b, double *out, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t want = (n + 255) / 256;
    const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
    k_rel_diff<<<blocks, 256, 0, s>>>(a, b, out, n);
    return cudaGetLastError();
}

}  // namespace rewl

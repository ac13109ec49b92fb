// Candidate clustering and coincidences on the GPU (Sec. "Candidate clustering
// and coincidences", Eq. norm; App. "Theory of coincidences").
//
//   fh_cluster       single-linkage clusters of one candidate set: candidates
//                    whose distance (Eq. norm, in mean coarse-bin widths) is at
//                    most d_max are linked; every cluster is labelled by its
//                    smallest member
//   fh_coincidences  the coincident pairs of two sets: frequencies referred to a
//                    common time, every parameter within its window in bins
//
// Both bucket candidates by frequency: a bucket is at least as wide as the
// largest frequency difference a link (or a coincidence) allows, d_max
// max(df) (w_f max(df)), so a candidate's partners lie in its own bucket and
// the two beside it.  Buckets are built by a count, the shared exclusive scan
// and a scatter.
//
// Clustering links each candidate to the larger-index candidates of those
// buckets through a lock-free union-find: a root is only ever hung below a
// smaller root (one compare-and-swap), so the root of every cluster is its
// smallest member and the labels do not depend on the order of the links.
// Coincidences count each set-1 candidate's partners, scan the counts into
// output offsets, then write the partners and sort each candidate's short list
// by index, so the pairs come out in (i, j) order.
//
// Arithmetic: every k and the distance are the binary64 operations of the
// definition in the order written (|x2 - x1|, 2 pi - that above pi for
// longitudes, divided by (w1 + w2) * 0.5; ((k_l^2 + k_b^2) + k_f^2) + k_fd^2 and
// its square root), so every link and every coincidence is decided exactly as
// the definition decides it.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fh_internal.h"

namespace fh {
namespace {

constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 6.283185307179586;
constexpr int kMaxBuckets = 1 << 22;
constexpr int kUnionLimit = 1 << 20;  // retries of one union (each follows another's progress)

__device__ __forceinline__ double bins_apart(double x1, double x2, double w1, double w2,
                                             bool wrap)
{
    double a = fabs(__dsub_rn(x2, x1));
    if (wrap && a > kPi) a = __dsub_rn(kTwoPi, a);
    return __ddiv_rn(a, __dmul_rn(__dadd_rn(w1, w2), 0.5));
}

__device__ __forceinline__ double norm_distance(const fh_cand_params &a, const fh_cand_params &b,
                                                double fa, double fb)
{
    const double kl = bins_apart(a.lam, b.lam, a.dlam, b.dlam, true);
    const double kb = bins_apart(a.beta, b.beta, a.dbeta, b.dbeta, false);
    const double kf = bins_apart(fa, fb, a.df, b.df, false);
    const double kd = bins_apart(a.fdot, b.fdot, a.dfdot, b.dfdot, false);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(kl, kl), __dmul_rn(kb, kb)),
                                          __dmul_rn(kf, kf)),
                                __dmul_rn(kd, kd)));
}

// A pair farther apart in one parameter than `reach` bins cannot link or
// coincide: that k exceeds reach, and the distance is at least each k.  These
// rejects run in binary32, whose pipe is many times GB300's binary64 one, and
// multiply instead of dividing; the exact binary64 divisions and square root
// are left to the few pairs that pass all four.
// A value rounded to float is off by at most half a float ulp, and the float
// difference of two such values by another, so |x2 - x1| >= the float
// difference - 2 ulp (ulp bounded by 2^-23 |x| plus the smallest normal); the
// width sum and the product carry relative errors of a few 2^-24, covered by
// the factor 1 + 1e-5.  A pair rejected here is rejected by the exact test;
// infinities and NaN never reject.
__device__ __forceinline__ float ulp2(float x) { return fabsf(x) * 2.4e-7f + 2.4e-38f; }
__device__ __forceinline__ bool far32(double xa, double xb, double wa, double wb, float reach)
{
    const float a = (float)xa, b = (float)xb;
    const float lim = reach * (((float)wa + (float)wb) * 0.5f) * 1.00001f;
    return fabsf(a - b) - 2.0f * ulp2(fmaxf(fabsf(a), fabsf(b))) > lim;
}
__device__ __forceinline__ bool lam_far32(double la, double lb, double wa, double wb, float reach)
{
    const float a0 = (float)la, b0 = (float)lb;
    float a = fabsf(a0 - b0);
    if (a > 3.14159265f) a = 6.28318531f - a;
    const float lim = reach * (((float)wa + (float)wb) * 0.5f) * 1.00001f;
    // near a difference of pi the two sides of the wrap differ by twice the
    // error of a, and the float constants by a few 1e-7
    return a - 4.0f * ulp2(fmaxf(fmaxf(fabsf(a0), fabsf(b0)), 6.3f)) - 1e-6f > lim;
}
// all four, evaluated without branches so that the lanes of a warp stay together
__device__ __forceinline__ bool any_far32(const fh_cand_params &a, const fh_cand_params &b,
                                          double fa, double fb, float reach_f, float reach_d,
                                          float reach_b, float reach_l)
{
    const bool r = far32(fa, fb, a.df, b.df, reach_f) | far32(a.fdot, b.fdot, a.dfdot, b.dfdot,
                                                              reach_d) |
                   far32(a.beta, b.beta, a.dbeta, b.dbeta, reach_b) |
                   lam_far32(a.lam, b.lam, a.dlam, b.dlam, reach_l);
    return r;
}

// order-preserving map of doubles to unsigned 64-bit keys (for atomic min / max)
__device__ __forceinline__ unsigned long long okey(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double from_okey(unsigned long long k)
{
    const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}

__device__ __forceinline__ bool cand_ok(const fh_cand_params &c)
{
    return isfinite(c.lam) && isfinite(c.beta) && isfinite(c.f) && isfinite(c.fdot) &&
           c.dlam > 0.0 && c.dbeta > 0.0 && c.df > 0.0 && c.dfdot > 0.0 && isfinite(c.dlam) &&
           isfinite(c.dbeta) && isfinite(c.df) && isfinite(c.dfdot);
}

// Range of the (shifted) frequencies and the largest frequency width.  rng:
// [0] okey(min f), [1] okey(max f), [2] okey(max df).  Non-finite values or
// widths <= 0 are flagged.
__global__ void range_kernel(const fh_cand_params *c, const double *fs, int32_t n,
                             unsigned long long *rng, int32_t *err, bool widths_only)
{
    unsigned long long lo = ~0ull, hi = 0ull, wd = 0ull;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const fh_cand_params x = c[i];
        bad = bad || !cand_ok(x);
        const double f = fs ? fs[i] : x.f;
        if (!widths_only) {
            lo = min(lo, okey(f));
            hi = max(hi, okey(f));
        }
        wd = max(wd, okey(x.df));
    }
    // one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        wd = max(wd, __shfl_xor_sync(0xffffffffu, wd, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (!widths_only) {
            atomicMin(rng + 0, lo);
            atomicMax(rng + 1, hi);
        }
        atomicMax(rng + 2, wd);
        if (bad) atomicOr(err, kErrInvalid);
    }
}

// bucket width: at least `reach` x max(df) (the largest frequency difference a
// link or a coincidence allows) and wide enough for nb buckets to span the
// range; 1e-6 wider so that two frequencies one width apart never land two
// buckets apart after rounding
struct Buckets {
    double f0, w;
    int32_t nb;
    __device__ __forceinline__ long long raw(double f) const
    {
        const double x = floor(__ddiv_rn(__dsub_rn(f, f0), w));
        return x < -1.0 ? -2 : (x > (double)nb ? (long long)nb + 1 : (long long)x);
    }
};

__global__ void bucket_setup_kernel(const unsigned long long *rng, int32_t nb, double reach,
                                    const unsigned long long *rng_w, Buckets *out)
{
    const double lo = from_okey(rng[0]), hi = from_okey(rng[1]);
    const double wd = from_okey(rng_w[2]);
    // an infinite width (an enormous window) puts everything in one bucket,
    // which is right; zero or NaN (no candidates, degenerate input) takes 1
    double w = fmax(reach * wd, (hi - lo) / (double)nb);
    if (!(w > 0.0)) w = 1.0;
    Buckets b;
    b.f0 = isfinite(lo) ? lo : 0.0;
    b.w = w * (1.0 + 1e-6);
    b.nb = nb;
    *out = b;
}

__global__ void bucket_count_kernel(const double *fs, int32_t n, const Buckets *bk, int32_t *bkt,
                                    int32_t *cnt)
{
    const Buckets b = *bk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long r = b.raw(fs[i]);
        const int32_t q = (int32_t)min(max(r, 0ll), (long long)b.nb - 1);
        bkt[i] = q;
        atomicAdd(cnt + q, 1);
    }
}

__global__ void bucket_scatter_kernel(const int32_t *bkt, int32_t n, const int64_t *start,
                                      int32_t *cursor, int32_t *order)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t q = bkt[i];
        order[start[q] + atomicAdd(cursor + q, 1)] = i;
    }
}

// ---------------------------------------------------------------- clustering
__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x, int32_t *err)
{
    for (int it = 0; it < kUnionLimit; ++it) {
        const int32_t p = ((volatile int32_t *)parent)[x];
        if (p == x) return x;
        const int32_t gp = ((volatile int32_t *)parent)[p];
        if (gp != p) atomicCAS(parent + x, p, gp);  // path halving: point to an ancestor
        x = gp;
    }
    atomicOr(err, kErrRange);
    return x;
}

__device__ __forceinline__ void uf_union(int32_t *parent, int32_t a, int32_t b, int32_t *err)
{
    for (int it = 0; it < kUnionLimit; ++it) {
        const int32_t ra = uf_find(parent, a, err), rb = uf_find(parent, b, err);
        if (ra == rb) return;
        const int32_t lo = min(ra, rb), hi = max(ra, rb);
        // hang the larger root below the smaller one, unless it stopped being a root
        if (atomicCAS(parent + hi, hi, lo) == hi) return;
        a = lo;
        b = hi;
    }
    atomicOr(err, kErrRange);
}

// threads take the candidates in bucket order, so the lanes of a warp scan
// the same buckets
__global__ void link_kernel(const fh_cand_params *c, int32_t n, double d_max, const int32_t *bkt,
                            const int64_t *start, const int32_t *order, int32_t nb,
                            int32_t *parent, int32_t *err)
{
    const float dm32 = (float)d_max;  // rounds to nearest: the 1e-5 factor covers it
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int32_t i = order[t];
        const fh_cand_params a = c[i];
        const int32_t q = bkt[i];
        for (int32_t qq = max(q - 1, 0); qq <= min(q + 1, nb - 1); ++qq) {
            for (int64_t p = start[qq]; p < start[qq + 1]; ++p) {
                const int32_t j = order[p];
                if (j <= i) continue;
                const fh_cand_params b = c[j];
                if (any_far32(a, b, a.f, b.f, dm32, dm32, dm32, dm32)) continue;
                if (norm_distance(a, b, a.f, b.f) <= d_max) uf_union(parent, i, j, err);
            }
        }
    }
}

__global__ void init_parent_kernel(int32_t *parent, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        parent[i] = i;
}

__global__ void finish_labels_kernel(int32_t *parent, int32_t n, int32_t *label,
                                     int32_t *n_roots, int32_t *err)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t r = uf_find(parent, i, err);
        label[i] = r;
        if (r == i) atomicAdd(n_roots, 1);
    }
}

// ---------------------------------------------------------------- coincidences
__global__ void shift_kernel(const fh_cand_params *c, int32_t n, double dt, double *fs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        fs[i] = __dadd_rn(c[i].f, __dmul_rn(c[i].fdot, dt));
}

struct CoinArgs {
    const fh_cand_params *c1, *c2;
    const double *f1, *f2;
    int32_t n1, n2;
    double w_lam, w_beta, w_f, w_fdot;
    const Buckets *bk;
    const int64_t *start;
    const int32_t *order;
    const int32_t *order1;  // set 1 in the order of set 2's buckets
};

// every window must hold; frequency first (with its cheap reject), then the rest
__device__ __forceinline__ bool coincide(const CoinArgs &a, const fh_cand_params &x, double fx,
                                         int32_t j)
{
    const double fy = a.f2[j];
    const fh_cand_params y = a.c2[j];
    if (any_far32(x, y, fx, fy, (float)a.w_f, (float)a.w_fdot, (float)a.w_beta,
                  (float)a.w_lam))
        return false;
    return bins_apart(fx, fy, x.df, y.df, false) <= a.w_f &&
           bins_apart(x.fdot, y.fdot, x.dfdot, y.dfdot, false) <= a.w_fdot &&
           bins_apart(x.beta, y.beta, x.dbeta, y.dbeta, false) <= a.w_beta &&
           bins_apart(x.lam, y.lam, x.dlam, y.dlam, true) <= a.w_lam;
}

__global__ void coin_count_kernel(const CoinArgs a, int32_t *cnt1, int32_t *cnt2)
{
    const Buckets b = *a.bk;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.n1; t += gridDim.x * blockDim.x) {
        const int32_t i = a.order1[t];
        const fh_cand_params x = a.c1[i];
        const double fx = a.f1[i];
        const long long r = b.raw(fx);
        int c = 0;
        for (long long qq = max(r - 1, 0ll); qq <= min(r + 1, (long long)b.nb - 1); ++qq)
            for (int64_t p = a.start[qq]; p < a.start[qq + 1]; ++p) {
                const int32_t j = a.order[p];
                if (coincide(a, x, fx, j)) {
                    ++c;
                    if (cnt2) atomicAdd(cnt2 + j, 1);
                }
            }
        cnt1[i] = c;
    }
}

__global__ void coin_write_kernel(const CoinArgs a, const int64_t *off, int64_t capacity,
                                  int32_t *pairs)
{
    const Buckets b = *a.bk;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.n1; t += gridDim.x * blockDim.x) {
        const int32_t i = a.order1[t];
        const fh_cand_params x = a.c1[i];
        const double fx = a.f1[i];
        const long long r = b.raw(fx);
        const int64_t o0 = off[i];
        int64_t o = o0;
        for (long long qq = max(r - 1, 0ll); qq <= min(r + 1, (long long)b.nb - 1); ++qq)
            for (int64_t p = a.start[qq]; p < a.start[qq + 1]; ++p) {
                const int32_t j = a.order[p];
                if (coincide(a, x, fx, j)) {
                    if (o < capacity) {
                        // insertion into the candidate's list, kept sorted by j
                        int64_t q = o;
                        while (q > o0 && pairs[2 * (q - 1) + 1] > j) {
                            pairs[2 * q] = i;
                            pairs[2 * q + 1] = pairs[2 * (q - 1) + 1];
                            --q;
                        }
                        pairs[2 * q] = i;
                        pairs[2 * q + 1] = j;
                    }
                    ++o;
                }
            }
    }
}

// ---------------------------------------------------------------- cluster coincidences
// Each coincident pair of clusters keeps its nearest coincident pair.  A hash
// table (open addressing, 64-bit keys cluster1 << 32 | cluster2, twice as many
// slots as pairs) gives every pair of clusters a slot; the slot keeps the
// smallest distance (atomic minimum of the bits of a non-negative double, which
// order like the values) and then the smallest pair index at that distance.
// The pairs come in (i, j) order, so the representatives, compacted in pair
// order, come out in (i, j) order too.
constexpr unsigned long long kEmptyKey = ~0ull;

struct CCArgs {
    const fh_cand_params *c1, *c2;
    const int32_t *label1, *label2, *pairs;
    int32_t n1, n2;
    int64_t n_pairs;
    double dt1, dt2;  // t_c - t_ref of each set
    unsigned long long *keys, *dmin, *best;
    int64_t tmask;
    int32_t *slot, *flag;
    double *dist;
    int32_t *err;
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void cc_insert_kernel(const CCArgs a)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = a.pairs[2 * p], j = a.pairs[2 * p + 1];
        bool ok = i >= 0 && i < a.n1 && j >= 0 && j < a.n2;
        if (ok && p > 0) {
            const int32_t pi = a.pairs[2 * p - 2], pj = a.pairs[2 * p - 1];
            ok = pi < i || (pi == i && pj < j);  // strictly increasing (i, j)
        }
        const int32_t la = ok ? a.label1[i] : -1, lb = ok ? a.label2[j] : -1;
        ok = ok && la >= 0 && la < a.n1 && lb >= 0 && lb < a.n2;
        if (!ok) {
            atomicOr(a.err, kErrInvalid);
            a.slot[p] = -1;
            continue;
        }
        const unsigned long long key = ((unsigned long long)(uint32_t)la << 32) | (uint32_t)lb;
        int64_t h = (int64_t)(mix64(key) & (unsigned long long)a.tmask);
        int32_t at = -1;
        for (int64_t it = 0; it <= a.tmask; ++it) {  // the table is at most half full
            const unsigned long long old = atomicCAS(a.keys + h, kEmptyKey, key);
            if (old == kEmptyKey || old == key) {
                at = (int32_t)h;
                break;
            }
            h = (h + 1) & a.tmask;
        }
        if (at < 0) {
            atomicOr(a.err, kErrRange);
            a.slot[p] = -1;
            continue;
        }
        const fh_cand_params x = a.c1[i], y = a.c2[j];
        const double fx = __dadd_rn(x.f, __dmul_rn(x.fdot, a.dt1));
        const double fy = __dadd_rn(y.f, __dmul_rn(y.fdot, a.dt2));
        const double d = norm_distance(x, y, fx, fy);
        a.dist[p] = d;
        a.slot[p] = at;
        atomicMin(a.dmin + at, (unsigned long long)__double_as_longlong(d));
    }
}

__global__ void cc_best_kernel(const CCArgs a)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t h = a.slot[p];
        if (h >= 0 &&
            (unsigned long long)__double_as_longlong(a.dist[p]) == a.dmin[h])
            atomicMin(a.best + h, (unsigned long long)p);
    }
}

__global__ void cc_flag_kernel(const CCArgs a)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t h = a.slot[p];
        a.flag[p] = (h >= 0 && a.best[h] == (unsigned long long)p) ? 1 : 0;
    }
}

__global__ void cc_write_kernel(const CCArgs a, const int64_t *off, int64_t capacity,
                                int32_t *out, double *out_d)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (!a.flag[p]) continue;
        const int64_t k = off[p];
        if (k >= capacity) continue;
        const int32_t i = a.pairs[2 * p], j = a.pairs[2 * p + 1];
        out[4 * k] = a.label1[i];
        out[4 * k + 1] = a.label2[j];
        out[4 * k + 2] = i;
        out[4 * k + 3] = j;
        if (out_d) out_d[k] = a.dist[p];
    }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

// buckets of n candidates by the frequencies fs: bkt, start (nb + 1), order
cudaError_t build_buckets(const double *fs, int32_t n, int32_t nb, const Buckets *bk,
                          int32_t *bkt, int64_t *start, int32_t *order, Scratch &sc,
                          cudaStream_t s)
{
    int32_t *cnt = nullptr, *cursor = nullptr;
    cudaError_t e = sc.get(&cnt, (size_t)nb);
    if (e == cudaSuccess) e = sc.get(&cursor, (size_t)nb);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * (size_t)nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, 4 * (size_t)nb, s);
    if (e == cudaSuccess && n > 0) {
        bucket_count_kernel<<<grid_for(n), 256, 0, s>>>(fs, n, bk, bkt, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_exclusive_scan(cnt, nb, start, 1, nullptr, s);
    if (e == cudaSuccess && n > 0) {
        bucket_scatter_kernel<<<grid_for(n), 256, 0, s>>>(bkt, n, start, cursor, order);
        e = cudaGetLastError();
    }
    return e;
}

int report(int32_t h_err)
{
    if (h_err & kErrInvalid)
        return set_error(FH_ERR_INVALID_ARG, "a candidate value is not finite or a width <= 0");
    if (h_err & kErrRange) return set_error(FH_ERR_TIMEOUT, "union-find retry limit reached");
    return FH_OK;
}

}  // namespace
}  // namespace fh

using namespace fh;

extern "C" {

int fh_cluster(const fh_cand_params *cands, int32_t n, double d_max, int32_t *label,
               int32_t *n_clusters, void *stream)
{
    if ((n > 0 && (!cands || !label)) || !n_clusters || n < 0 || n > (1 << 30) ||
        !(d_max >= 0.0) || !std::isfinite(d_max))
        return set_error(FH_ERR_INVALID_ARG, "need cands, label, n in [0, 2^30], finite d_max >= 0");
    *n_clusters = 0;
    if (n == 0) return FH_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc(s);
    const int32_t nb = std::min(n, kMaxBuckets);
    unsigned long long *rng = nullptr;
    Buckets *bk = nullptr;
    double *fs = nullptr;
    int32_t *bkt = nullptr, *order = nullptr, *parent = nullptr, *err = nullptr, *roots = nullptr;
    int64_t *start = nullptr;
    cudaError_t e = sc.get(&rng, 3);
    if (e == cudaSuccess) e = sc.get(&bk, 1);
    if (e == cudaSuccess) e = sc.get(&fs, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&bkt, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&order, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&parent, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&err, 2);
    if (e == cudaSuccess) e = sc.get(&start, (size_t)nb + 1);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (cluster)");
    roots = err + 1;
    const unsigned long long init[3] = {~0ull, 0ull, 0ull};
    e = cudaMemcpyAsync(rng, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 8, s);
    if (e == cudaSuccess) {
        range_kernel<<<grid_for(n), 256, 0, s>>>(cands, nullptr, n, rng, err, false);
        shift_kernel<<<grid_for(n), 256, 0, s>>>(cands, n, 0.0, fs);  // f itself (f + fdot 0)
        bucket_setup_kernel<<<1, 1, 0, s>>>(rng, nb, d_max, rng, bk);
        init_parent_kernel<<<grid_for(n), 256, 0, s>>>(parent, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = build_buckets(fs, n, nb, bk, bkt, start, order, sc, s);
    if (e == cudaSuccess) {
        link_kernel<<<grid_for(n), 256, 0, s>>>(cands, n, d_max, bkt, start, order, nb, parent,
                                                 err);
        finish_labels_kernel<<<grid_for(n), 256, 0, s>>>(parent, n, label, roots, err);
        e = cudaGetLastError();
    }
    int32_t h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, err, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cluster");
    *n_clusters = h[1];
    return report(h[0]);
}

int fh_coincidences(const fh_cand_params *c1, int32_t n1, double t_ref1,
                    const fh_cand_params *c2, int32_t n2, double t_ref2, double t_c,
                    const double *win, int32_t *pairs, int64_t capacity, int64_t *n_pairs,
                    int32_t *n_match1, int32_t *n_match2, void *stream)
{
    if ((n1 > 0 && !c1) || (n2 > 0 && !c2) || !win || !n_pairs || (capacity > 0 && !pairs) ||
        n1 < 0 || n2 < 0 || n1 > (1 << 30) || n2 > (1 << 30) || capacity < 0)
        return set_error(FH_ERR_INVALID_ARG, "bad candidate sets or outputs");
    for (int q = 0; q < 4; ++q)
        if (!(win[q] >= 0.0) || !std::isfinite(win[q]))
            return set_error(FH_ERR_INVALID_ARG, "windows must be finite and >= 0");
    if (!std::isfinite(t_ref1) || !std::isfinite(t_ref2) || !std::isfinite(t_c))
        return set_error(FH_ERR_INVALID_ARG, "reference times must be finite");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    *n_pairs = 0;
    cudaError_t e = cudaSuccess;
    if (n_match2 && n2 > 0) e = cudaMemsetAsync(n_match2, 0, 4 * (size_t)n2, s);
    if (e == cudaSuccess && n_match1 && n1 > 0 && n2 == 0)
        e = cudaMemsetAsync(n_match1, 0, 4 * (size_t)n1, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync (coincidences)");
    if (n1 == 0 || n2 == 0) {
        e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? FH_OK : cuda_error(e, "coincidences");
    }
    Scratch sc(s);
    const int32_t nb = std::min(n2, kMaxBuckets);
    unsigned long long *rng = nullptr, *rngw = nullptr;
    Buckets *bk = nullptr;
    double *f1 = nullptr, *f2 = nullptr;
    int32_t *bkt = nullptr, *order = nullptr, *err = nullptr, *cnt1 = nullptr;
    int64_t *start = nullptr, *off = nullptr;
    e = sc.get(&rng, 3);
    if (e == cudaSuccess) e = sc.get(&rngw, 3);
    if (e == cudaSuccess) e = sc.get(&bk, 1);
    if (e == cudaSuccess) e = sc.get(&f1, (size_t)n1);
    if (e == cudaSuccess) e = sc.get(&f2, (size_t)n2);
    if (e == cudaSuccess) e = sc.get(&bkt, (size_t)n2);
    if (e == cudaSuccess) e = sc.get(&order, (size_t)n2);
    if (e == cudaSuccess) e = sc.get(&err, 1);
    if (e == cudaSuccess) e = sc.get(&start, (size_t)nb + 1);
    if (e == cudaSuccess) e = sc.get(&off, (size_t)n1 + 1);
    if (e == cudaSuccess) {
        if (n_match1)
            cnt1 = n_match1;
        else
            e = sc.get(&cnt1, (size_t)n1);
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (coincidences)");
    const unsigned long long init[3] = {~0ull, 0ull, 0ull};
    e = cudaMemcpyAsync(rng, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rngw, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    if (e == cudaSuccess) {
        // frequencies at the common time: f + fdot (t_c - t_ref)
        shift_kernel<<<grid_for(n1), 256, 0, s>>>(c1, n1, t_c - t_ref1, f1);
        shift_kernel<<<grid_for(n2), 256, 0, s>>>(c2, n2, t_c - t_ref2, f2);
        range_kernel<<<grid_for(n2), 256, 0, s>>>(c2, f2, n2, rng, err, false);
        range_kernel<<<grid_for(n1), 256, 0, s>>>(c1, f1, n1, rngw, err, true);
        range_kernel<<<grid_for(n2), 256, 0, s>>>(c2, f2, n2, rngw, err, true);
        bucket_setup_kernel<<<1, 1, 0, s>>>(rng, nb, win[2], rngw, bk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = build_buckets(f2, n2, nb, bk, bkt, start, order, sc, s);
    // set 1 sorted by the same buckets (clamped), so that a warp's threads scan
    // the same part of set 2
    int32_t *bkt1 = nullptr, *order1 = nullptr;
    int64_t *start1 = nullptr;
    if (e == cudaSuccess) e = sc.get(&bkt1, (size_t)n1);
    if (e == cudaSuccess) e = sc.get(&order1, (size_t)n1);
    if (e == cudaSuccess) e = sc.get(&start1, (size_t)nb + 1);
    if (e == cudaSuccess) e = build_buckets(f1, n1, nb, bk, bkt1, start1, order1, sc, s);
    CoinArgs a{c1, c2, f1, f2, n1, n2, win[0], win[1], win[2], win[3], bk, start, order, order1};
    if (e == cudaSuccess) {
        coin_count_kernel<<<grid_for(n1), 256, 0, s>>>(a, cnt1, n_match2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_exclusive_scan(cnt1, n1, off, 1, nullptr, s);
    if (e == cudaSuccess && capacity > 0) {
        coin_write_kernel<<<grid_for(n1), 256, 0, s>>>(a, off, capacity, pairs);
        e = cudaGetLastError();
    }
    int64_t total = 0;
    int32_t h_err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, off + n1, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "coincidences");
    const int rc = report(h_err);
    if (rc) return rc;
    *n_pairs = total;
    if (total > capacity)
        return set_error(FH_ERR_CAPACITY, "%lld coincident pairs, capacity %lld",
                         (long long)total, (long long)capacity);
    return FH_OK;
}

int fh_cluster_coincidences(const fh_cand_params *c1, int32_t n1, double t_ref1,
                            const int32_t *label1, const fh_cand_params *c2, int32_t n2,
                            double t_ref2, const int32_t *label2, double t_c,
                            const int32_t *pairs, int64_t n_pairs, int32_t *out, double *out_d,
                            int64_t capacity, int64_t *n_out, void *stream)
{
    if (!n_out || n_pairs < 0 || n_pairs > ((int64_t)1 << 30) || capacity < 0 || n1 < 0 ||
        n2 < 0 || (n_pairs > 0 && (!c1 || !c2 || !label1 || !label2 || !pairs)) ||
        (capacity > 0 && !out))
        return set_error(FH_ERR_INVALID_ARG, "bad candidate sets, labels, pairs or outputs");
    if (!std::isfinite(t_ref1) || !std::isfinite(t_ref2) || !std::isfinite(t_c))
        return set_error(FH_ERR_INVALID_ARG, "reference times must be finite");
    *n_out = 0;
    if (n_pairs == 0) return FH_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc(s);
    int64_t tsize = 2;
    while (tsize < 2 * n_pairs) tsize <<= 1;
    unsigned long long *keys = nullptr, *dmin = nullptr, *best = nullptr;
    int32_t *slot = nullptr, *flag = nullptr, *err = nullptr;
    double *dist = nullptr;
    int64_t *off = nullptr;
    cudaError_t e = sc.get(&keys, (size_t)tsize);
    if (e == cudaSuccess) e = sc.get(&dmin, (size_t)tsize);
    if (e == cudaSuccess) e = sc.get(&best, (size_t)tsize);
    if (e == cudaSuccess) e = sc.get(&slot, (size_t)n_pairs);
    if (e == cudaSuccess) e = sc.get(&flag, (size_t)n_pairs);
    if (e == cudaSuccess) e = sc.get(&dist, (size_t)n_pairs);
    if (e == cudaSuccess) e = sc.get(&off, (size_t)n_pairs + 1);
    if (e == cudaSuccess) e = sc.get(&err, 1);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (cluster coincidences)");
    e = cudaMemsetAsync(keys, 0xFF, 8 * (size_t)tsize, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmin, 0xFF, 8 * (size_t)tsize, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(best, 0xFF, 8 * (size_t)tsize, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    CCArgs a{c1, c2, label1, label2, pairs, n1, n2, n_pairs, t_c - t_ref1, t_c - t_ref2,
             keys, dmin, best, tsize - 1, slot, flag, dist, err};
    const int grid = grid_for(n_pairs);
    if (e == cudaSuccess) {
        cc_insert_kernel<<<grid, 256, 0, s>>>(a);
        cc_best_kernel<<<grid, 256, 0, s>>>(a);
        cc_flag_kernel<<<grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_exclusive_scan(flag, n_pairs, off, 1, nullptr, s);
    if (e == cudaSuccess && capacity > 0) {
        cc_write_kernel<<<grid, 256, 0, s>>>(a, off, capacity, out, out_d);
        e = cudaGetLastError();
    }
    int64_t total = 0;
    int32_t h_err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, off + n_pairs, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cluster coincidences");
    if (h_err & kErrInvalid)
        return set_error(FH_ERR_INVALID_ARG, "pairs out of range or not in (i, j) order, or "
                                             "labels out of range");
    if (h_err) return set_error(FH_ERR_RANGE, "cluster-pair table full");
    *n_out = total;
    if (total > capacity)
        return set_error(FH_ERR_CAPACITY, "%lld cluster pairs, capacity %lld", (long long)total,
                         (long long)capacity);
    return FH_OK;
}

}  // extern "C"

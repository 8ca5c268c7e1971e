// lc_bucket.cu -- the rank-order replacement of one E13 iteration (Sec. 2.1
// third step, Sec. 3.2.2: x[perm[r]] = s[r] with perm the stable argsort of
// x_adj) as a sample sort: one bucket pass through HBM and one on-chip pass
// that ranks every element exactly.
//
// Per curve of N = 2^13 .. 2^18 FP32 samples:
//   k_bk_sample   1024 values of x_adj at a fixed stride, sorted in shared
//                 memory; 255 of them become the splitters of 256 buckets
//                 (bucket b holds spl[b-1] <= x < spl[b]);
//   k_bk_hist     per 2048-element tile: bucket of every element (binary
//                 search over the splitters) and the tile's bucket counts;
//                 the curve's minimum and maximum;
//   k_bk_scan     tile prefixes and bucket bases of the curve, and groups of
//                 consecutive buckets of at most kBkCap elements;
//   k_bk_scatter  every element (value, position | bucket << 24) into its
//                 tile's slice of its bucket (shared-memory atomics: the
//                 order inside a slice is arbitrary);
//   k_bk_finish   one group per block, in shared memory: each bucket is split
//                 into as many sub-buckets as it has elements by linear
//                 interpolation of the value between the bucket's bounds
//                 (monotone), the group is counting-sorted by sub-bucket, and
//                 every element is ranked among the members of its sub-bucket
//                 by (value, position) -- the stable argsort order, whatever
//                 order the scatter left.  rank = bucket base + rank in group;
//                 the block writes x[position] = s[rank].
// A bucket of more than kBkCap elements (a spike of equal or nearly equal
// values) is one group of its own, sorted by a block-level LSD radix sort on
// (value, position) through global memory instead.
//
// HBM bytes per element: 4 (histogram) + 4 + 8 (scatter) + 8 + 4 + 4 (finish)
// = 32, against 76 for the four 8-bit LSD passes and their histograms.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "lc_internal.h"

namespace lc {

constexpr int kBkBuckets = 256;
constexpr int kBkSample = 1024;
constexpr int kBkThreads = 512;                  // sample and finish kernels
constexpr int kBkPer = kBkCap / kBkThreads;      // elements per finish thread
constexpr int kBkTileThreads = 256;              // histogram and scatter kernels
constexpr int kBkTilePer = kSortTile / kBkTileThreads;  // 8 elements per thread and tile

// Per-curve words of the auxiliary area (u32): splitters (float bits), the
// curve's min and max (order keys), bucket bases (257), then the group count
// and the group starts (bucket indices, gmax + 1).
constexpr int kAuxSpl = 0;
constexpr int kAuxMin = 256;
constexpr int kAuxMax = 257;
constexpr int kAuxBase = 258;
constexpr int kAuxGcount = kAuxBase + kBkBuckets + 1;   // 515
constexpr int kAuxGstart = kAuxGcount + 1;              // 516

int bucket_gmax(uint32_t log2n)
{
    // greedy groups: any two consecutive ones hold more than kBkCap elements
    return 2 * (int)(((size_t)1 << log2n) / kBkCap) + 1;
}

size_t bucket_aux_words(uint32_t log2n)
{
    const size_t w = (size_t)kAuxGstart + (size_t)bucket_gmax(log2n) + 1;
    return (w + 63) / 64 * 64;
}

bool bucket_supported(lc_precision prec, uint32_t log2n)
{
    return prec == LC_FP32 && log2n >= kBkMinLog2 && log2n <= kBkMaxLog2;
}

bool bucket_enabled_from_env()
{
    const char* e = std::getenv("LC_SORT");
    return !(e && std::strcmp(e, "radix") == 0);
}

struct BkArgs {
    const int* cls_curves;
    const CurveDev* curves;
    const uint32_t* eff_iters;
    const int* d_iter;       // null: every curve active
    const float* xadj;       // values to rank (the inverse transform's output)
    uint32_t* aux;           // [ci][stride]
    uint32_t* hist;          // [ci][tpc][256]
    uint32_t* keys;          // bucket order: value bits
    uint32_t* vals;          // bucket order: position | bucket << 24
    uint32_t* keys2;         // ping-pong of the oversize-bucket sort
    uint32_t* vals2;
    const float* s;          // sorted draws
    float* x_out;            // x[position] = s[rank]
    int tpc;
    int stride;              // aux words per curve
    int gmax;
    uint32_t log2n;
};

__device__ __forceinline__ bool bk_active(const BkArgs& a, int c)
{
    return !a.d_iter || (uint32_t)(*a.d_iter) < a.eff_iters[c];
}

// Number of splitters <= v: the bucket of v (spl ascending, 255 entries used).
__device__ __forceinline__ uint32_t bucket_of(const float* spl, float v)
{
    uint32_t b = 0;
#pragma unroll
    for (uint32_t st = 128; st >= 1; st >>= 1)
        if (v >= spl[b + st - 1]) b += st;
    return b;
}

// ------------------------------------------------------------------ sample
__global__ void __launch_bounds__(kBkThreads) k_bk_sample(const BkArgs a)
{
    const int ci = blockIdx.x;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float sm[kBkSample];
    const int tid = threadIdx.x;
    const uint64_t off = a.curves[c].off;
    const uint32_t stride = (1u << a.log2n) / kBkSample;
    for (int i = tid; i < kBkSample; i += kBkThreads) sm[i] = a.xadj[off + (uint64_t)i * stride + stride / 2];
    __syncthreads();
    // bitonic sort, ascending; thread tid owns pair p = tid of every stage
    for (int k = 2; k <= kBkSample; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int i = 2 * j * (tid / j) + (tid % j);
            const int l = i + j;
            const bool up = (i & k) == 0;
            const float u = sm[i], v = sm[l];
            if ((u > v) == up) {
                sm[i] = v;
                sm[l] = u;
            }
            __syncthreads();
        }
    }
    uint32_t* A = a.aux + (size_t)ci * a.stride;
    if (tid < kBkBuckets - 1) A[kAuxSpl + tid] = __float_as_uint(sm[(kBkSample / kBkBuckets) * (tid + 1)]);
    if (tid == kBkBuckets - 1) A[kAuxSpl + tid] = 0x7f800000u;  // +inf, never compared
    if (tid == 0) {
        A[kAuxMin] = 0xffffffffu;
        A[kAuxMax] = 0u;
    }
}

// ------------------------------------------------------------------ histogram
template <int TPB>
__global__ void __launch_bounds__(kBkTileThreads) k_bk_hist(const BkArgs a)
{
    constexpr int W = kBkTileThreads / 32;
    constexpr int V4 = kSortTile / 4 / kBkTileThreads;  // float4 loads per thread and tile
    const int bpc = a.tpc / TPB;
    const int ci = blockIdx.x / bpc;
    const int t0 = (blockIdx.x % bpc) * TPB;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float spl[kBkBuckets];
    __shared__ uint32_t h[TPB][W][kBkBuckets];
    __shared__ uint32_t red[2][W];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* A = a.aux + (size_t)ci * a.stride;
    spl[tid] = __uint_as_float(A[kAuxSpl + tid]);
#pragma unroll
    for (int u = 0; u < TPB; ++u)
#pragma unroll
        for (int w = 0; w < W; ++w) h[u][w][tid] = 0;
    const uint64_t base = a.curves[c].off + (uint64_t)t0 * kSortTile;
    const float4* __restrict__ src = (const float4*)(a.xadj + base);
    float4 q[TPB * V4];
#pragma unroll
    for (int e = 0; e < TPB * V4; ++e) {
        const int u = e / V4, v = tid + (e % V4) * kBkTileThreads;
        q[e] = src[(size_t)u * (kSortTile / 4) + v];
    }
    __syncthreads();
    uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
    for (int e = 0; e < TPB * V4; ++e) {
        const int u = e / V4;
        const float vv[4] = {q[e].x, q[e].y, q[e].z, q[e].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            atomicAdd(&h[u][warp][bucket_of(spl, vv[j])], 1u);
            const uint32_t k = order_key(vv[j]);
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
        red[0][warp] = kmin;
        red[1][warp] = kmax;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPB; ++u) {
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cnt += h[u][w][tid];
        a.hist[((size_t)ci * a.tpc + t0 + u) * kBkBuckets + tid] = cnt;
    }
    if (tid == 0) {
        uint32_t m0 = red[0][0], m1 = red[1][0];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            m0 = min(m0, red[0][w]);
            m1 = max(m1, red[1][w]);
        }
        atomicMin(&A[kAuxMin], m0);
        atomicMax(&A[kAuxMax], m1);
    }
}

// ------------------------------------------------------------------ scan
// One block (256 threads, thread b = bucket b) per curve.
__global__ void __launch_bounds__(kBkBuckets) k_bk_scan(const BkArgs a)
{
    const int ci = blockIdx.x;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ uint32_t wsum[kBkBuckets / 32];
    __shared__ uint32_t cnt[kBkBuckets];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* h = a.hist + (size_t)ci * a.tpc * kBkBuckets + tid;
    uint32_t run = 0;
    for (int t0 = 0; t0 < a.tpc; t0 += 16) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = t0 + u < a.tpc ? h[(size_t)(t0 + u) * kBkBuckets] : 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (t0 + u < a.tpc) h[(size_t)(t0 + u) * kBkBuckets] = run;
            run += v[u];
        }
    }
    // exclusive scan of the bucket totals
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    cnt[tid] = run;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    uint32_t* A = a.aux + (size_t)ci * a.stride;
    A[kAuxBase + tid] = woff + incl - run;
    if (tid == kBkBuckets - 1) A[kAuxBase + kBkBuckets] = woff + incl;
    if (tid == 0) {
        // greedy groups of consecutive buckets holding at most kBkCap
        // elements; a larger bucket forms a group of its own
        uint32_t g = 0, acc = 0;
        A[kAuxGstart] = 0;
        for (int b = 0; b < kBkBuckets; ++b) {
            const uint32_t n = cnt[b];
            if (acc > 0 && acc + n > (uint32_t)kBkCap) {
                A[kAuxGstart + (++g)] = (uint32_t)b;
                acc = 0;
            }
            acc += n;
        }
        A[kAuxGstart + g + 1] = kBkBuckets;
        A[kAuxGcount] = g + 1;
    }
}

// ------------------------------------------------------------------ scatter
__global__ void __launch_bounds__(kBkTileThreads) k_bk_scatter(const BkArgs a)
{
    constexpr int V4 = kSortTile / 4 / kBkTileThreads;
    const int ci = blockIdx.x / a.tpc;
    const int t = blockIdx.x % a.tpc;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float spl[kBkBuckets];
    __shared__ uint32_t cur[kBkBuckets];
    const int tid = threadIdx.x;
    const uint32_t* A = a.aux + (size_t)ci * a.stride;
    spl[tid] = __uint_as_float(A[kAuxSpl + tid]);
    cur[tid] = a.hist[((size_t)ci * a.tpc + t) * kBkBuckets + tid] + A[kAuxBase + tid];
    const uint64_t off = a.curves[c].off;
    const uint32_t e0 = (uint32_t)t * kSortTile;
    const float4* __restrict__ src = (const float4*)(a.xadj + off + e0);
    float4 q[V4];
#pragma unroll
    for (int e = 0; e < V4; ++e) q[e] = src[tid + e * kBkTileThreads];
    __syncthreads();
    uint32_t* __restrict__ kd = a.keys + off;
    uint32_t* __restrict__ vd = a.vals + off;
#pragma unroll
    for (int e = 0; e < V4; ++e) {
        const float vv[4] = {q[e].x, q[e].y, q[e].z, q[e].w};
        const uint32_t i0 = e0 + 4u * (uint32_t)(tid + e * kBkTileThreads);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t b = bucket_of(spl, vv[j]);
            const uint32_t pos = atomicAdd(&cur[b], 1u);
            kd[pos] = __float_as_uint(vv[j]);
            vd[pos] = (i0 + (uint32_t)j) | (b << 24);
        }
    }
}

// ------------------------------------------------------------------ finish
// Block-wide exclusive scan of v (kBkThreads threads).
__device__ __forceinline__ uint32_t bk_block_scan(uint32_t v, uint32_t* wsum, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t woff = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kBkThreads / 32; ++w) {
        const uint32_t x = wsum[w];
        woff += w < warp ? x : 0u;
        tot += x;
    }
    __syncthreads();
    if (total) *total = tot;
    return woff + incl - v;
}

// One stable LSD pass of the block over n (key, val) pairs in global memory,
// by the byte `shift` of the position (val, bits 0..23) when !KEYB, else of
// the value's order key.  Returns false (nothing moved) when every element
// has the same digit.
template <bool KEYB>
__device__ bool bk_block_pass(const uint32_t* __restrict__ ik, const uint32_t* __restrict__ iv,
                              uint32_t* __restrict__ ok, uint32_t* __restrict__ ov, int n, int shift,
                              uint32_t* hist, uint32_t (*wc)[256], uint32_t* wsum)
{
    constexpr int W = kBkThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto digit = [&](uint32_t k, uint32_t v) -> uint32_t {
        return KEYB ? (order_key(__uint_as_float(k)) >> shift) & 255u : ((v & 0xffffffu) >> shift) & 255u;
    };
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kBkThreads) atomicAdd(&hist[digit(ik[i], iv[i])], 1u);
    __syncthreads();
    const bool one = tid < 256 && hist[tid] == (uint32_t)n;
    if (__syncthreads_or(one)) return false;
    uint32_t base = bk_block_scan(tid < 256 ? hist[tid] : 0u, wsum, nullptr);  // digit tid's base
    const uint32_t lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < n; c0 += kBkThreads) {
        for (int q = tid; q < W * 256; q += kBkThreads) (&wc[0][0])[q] = 0;
        __syncthreads();
        const int i = c0 + tid;
        const bool valid = i < n;
        uint32_t k = 0, v = 0, d = 256u + lane;
        if (valid) {
            k = ik[i];
            v = iv[i];
            d = digit(k, v);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d) & __ballot_sync(0xffffffffu, valid);
        const uint32_t below = __popc(peers & lt);
        if (valid && below == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;
        if (tid < 256) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t x = wc[w][tid];
                wc[w][tid] = base + tot;
                tot += x;
            }
        }
        __syncthreads();
        if (valid) {
            const uint32_t dst = wc[warp][d] + below;
            ok[dst] = k;
            ov[dst] = v;
        }
        base += tot;
        __syncthreads();
    }
    return true;
}

// Oversize bucket: sort its n pairs by (order key, position) with block LSD
// passes (position bytes first), then x[position] = s[e0 + r].
__device__ void bk_oversize(const BkArgs& a, uint64_t off, uint32_t e0, int n, uint32_t* smem_u32)
{
    uint32_t* hist = smem_u32;
    uint32_t(*wc)[256] = (uint32_t(*)[256])(smem_u32 + 256);
    uint32_t* wsum = smem_u32 + 256 + (kBkThreads / 32) * 256;
    uint32_t* k0 = a.keys + off + e0;
    uint32_t* v0 = a.vals + off + e0;
    uint32_t* k1 = a.keys2 + off + e0;
    uint32_t* v1 = a.vals2 + off + e0;
    bool in0 = true;
    const int npos = a.log2n > 16 ? 3 : 2;  // position bytes in use
    for (int q = 0; q < npos + 4; ++q) {
        const bool keyb = q >= npos;
        const int shift = 8 * (keyb ? q - npos : q);
        const uint32_t* ik = in0 ? k0 : k1;
        const uint32_t* iv = in0 ? v0 : v1;
        uint32_t* ok = in0 ? k1 : k0;
        uint32_t* ov = in0 ? v1 : v0;
        const bool moved = keyb ? bk_block_pass<true>(ik, iv, ok, ov, n, shift, hist, wc, wsum)
                                : bk_block_pass<false>(ik, iv, ok, ov, n, shift, hist, wc, wsum);
        if (moved) in0 = !in0;
    }
    const uint32_t* vf = in0 ? v0 : v1;
    const float* __restrict__ s = a.s + off + e0;
    float* __restrict__ x = a.x_out + off;
    for (int r = threadIdx.x; r < n; r += kBkThreads) x[vf[r] & 0xffffffu] = s[r];
}

__global__ void __launch_bounds__(kBkThreads, 2) k_bk_finish(const BkArgs a)
{
    const int ci = blockIdx.x / a.gmax;
    const int g = blockIdx.x % a.gmax;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    const uint32_t* A = a.aux + (size_t)ci * a.stride;
    if ((uint32_t)g >= A[kAuxGcount]) return;
    const uint32_t b0 = A[kAuxGstart + g], b1 = A[kAuxGstart + g + 1];
    const uint32_t e0 = A[kAuxBase + b0], e1 = A[kAuxBase + b1];
    const int n = (int)(e1 - e0);
    if (n == 0) return;
    const uint64_t off = a.curves[c].off;
    extern __shared__ __align__(16) uint32_t bsm[];
    if (n > kBkCap) {  // one bucket of nearly equal values
        bk_oversize(a, off, e0, n, bsm);
        return;
    }
    float* sk = (float*)bsm;                 // [kBkCap] values by sub-bucket
    uint32_t* si = bsm + kBkCap;             // [kBkCap] positions by sub-bucket, then by rank
    uint32_t* st = bsm + 2 * kBkCap;         // [kBkCap] sub-bucket counts, then starts
    uint32_t* en = bsm + 3 * kBkCap;         // [kBkCap] sub-bucket cursors, then ends
    float* plo = (float*)(bsm + 4 * kBkCap);           // [256] bucket lower bound
    float* psc = (float*)(bsm + 4 * kBkCap + 256);     // [256] sub-buckets per unit value
    uint32_t* poff = bsm + 4 * kBkCap + 512;           // [256] first sub-bucket of the bucket
    uint32_t* pcnt = bsm + 4 * kBkCap + 768;           // [256] elements of the bucket
    uint32_t* wsum = bsm + 4 * kBkCap + 1024;          // [16]
    const int tid = threadIdx.x;
    const int nb = (int)(b1 - b0);
    for (int i = tid; i < nb; i += kBkThreads) {
        const uint32_t b = b0 + (uint32_t)i;
        const float lo = b == 0 ? key_value(A[kAuxMin]) : __uint_as_float(A[kAuxSpl + b - 1]);
        const float hi = b == kBkBuckets - 1 ? key_value(A[kAuxMax]) : __uint_as_float(A[kAuxSpl + b]);
        const uint32_t cb = A[kAuxBase + b + 1] - A[kAuxBase + b];
        const float d = hi - lo;
        plo[i] = lo;
        psc[i] = (d > 0.0f && cb > 0u) ? (float)cb / d : 0.0f;
        poff[i] = A[kAuxBase + b] - e0;
        pcnt[i] = cb;
    }
    for (int i = tid; i < kBkCap; i += kBkThreads) st[i] = 0u;
    __syncthreads();
    // load; sub-bucket of every element (monotone in the value inside a bucket)
    const uint32_t* __restrict__ kin = a.keys + off + e0;
    const uint32_t* __restrict__ vin = a.vals + off + e0;
    float key[kBkPer];
    uint32_t pos[kBkPer], sub[kBkPer];
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int p = tid + j * kBkThreads;
        if (p < n) {
            key[j] = __uint_as_float(kin[p]);
            pos[j] = vin[p];
        }
    }
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int p = tid + j * kBkThreads;
        if (p < n) {
            const uint32_t bl = min((pos[j] >> 24) - b0, (uint32_t)nb - 1u);
            pos[j] &= 0xffffffu;
            const float f = (key[j] - plo[bl]) * psc[bl];
            int sb = __float2int_rz(f);  // NaN -> 0
            sb = max(0, min(sb, (int)pcnt[bl] - 1));
            sub[j] = poff[bl] + (uint32_t)sb;
            atomicAdd(&st[sub[j]], 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the n sub-bucket counts: thread tid owns kBkPer consecutive ones
    {
        uint32_t v[kBkPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kBkPer; ++j) {
            const int q = tid * kBkPer + j;
            v[j] = q < n ? st[q] : 0u;
            sum += v[j];
        }
        uint32_t run = bk_block_scan(sum, wsum, nullptr);
#pragma unroll
        for (int j = 0; j < kBkPer; ++j) {
            const int q = tid * kBkPer + j;
            if (q < n) {
                st[q] = run;
                en[q] = run;
            }
            run += v[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int p = tid + j * kBkThreads;
        if (p < n) {
            const uint32_t q = atomicAdd(&en[sub[j]], 1u);
            sk[q] = key[j];
            si[q] = pos[j];
        }
    }
    __syncthreads();
    // rank among the sub-bucket's members by (value, position)
    uint32_t lr[kBkPer];
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int p = tid + j * kBkThreads;
        if (p < n) {
            const uint32_t s0 = st[sub[j]], s1 = en[sub[j]];
            uint32_t r = s0;
            for (uint32_t q = s0; q < s1; ++q) {
                const float kq = sk[q];
                r += (kq < key[j] || (kq == key[j] && si[q] < pos[j])) ? 1u : 0u;
            }
            lr[j] = r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBkPer; ++j)
        if (tid + j * kBkThreads < n) si[lr[j]] = pos[j];
    __syncthreads();
    const float* __restrict__ s = a.s + off + e0;
    float* __restrict__ x = a.x_out + off;
    float sv[kBkPer];
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int r = tid + j * kBkThreads;
        if (r < n) sv[j] = s[r];
    }
#pragma unroll
    for (int j = 0; j < kBkPer; ++j) {
        const int r = tid + j * kBkThreads;
        if (r < n) x[si[r]] = sv[j];
    }
}

constexpr size_t kBkFinishSmem = (size_t)(4 * kBkCap + 1024 + 32) * 4;

cudaError_t bucket_kernel_attributes()
{
    return cudaFuncSetAttribute(k_bk_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBkFinishSmem);
}

void launch_bucket_argsort(const Plan& p, const ClassInfo& k, const void* src, void* x_out, bool gated,
                           cudaStream_t st, uint64_t* launches, KernelTimes* kt)
{
    BkArgs a{};
    a.cls_curves = k.d_curves;
    a.curves = p.d_curves;
    a.eff_iters = p.d_eff_iters;
    a.d_iter = gated ? p.d_iter : nullptr;
    a.xadj = (const float*)src;
    a.aux = k.d_aux;
    a.hist = p.d_hist + k.hist_off;
    a.keys = (uint32_t*)p.d_keysA;
    a.vals = p.d_valsA;
    a.keys2 = (uint32_t*)p.d_f;
    a.vals2 = p.d_valsB;
    a.s = (const float*)p.d_s;
    a.x_out = (float*)(x_out ? x_out : p.d_x);
    a.tpc = k.tiles_per_curve;
    a.stride = (int)bucket_aux_words(k.log2n);
    a.gmax = bucket_gmax(k.log2n);
    a.log2n = k.log2n;
    if (kt) kt->begin(kGroupSortHistScan, st);
    k_bk_sample<<<k.ncurves, kBkThreads, 0, st>>>(a);
    const int tpb = std::min(4, a.tpc);
    if (tpb >= 4) k_bk_hist<4><<<k.ncurves * (a.tpc / 4), kBkTileThreads, 0, st>>>(a);
    else if (tpb >= 2) k_bk_hist<2><<<k.ncurves * (a.tpc / 2), kBkTileThreads, 0, st>>>(a);
    else k_bk_hist<1><<<k.ncurves * a.tpc, kBkTileThreads, 0, st>>>(a);
    k_bk_scan<<<k.ncurves, kBkBuckets, 0, st>>>(a);
    if (kt) kt->end(st);
    if (kt) kt->begin(kGroupSortScatter, st);
    k_bk_scatter<<<k.ncurves * a.tpc, kBkTileThreads, 0, st>>>(a);
    k_bk_finish<<<k.ncurves * a.gmax, kBkThreads, kBkFinishSmem, st>>>(a);
    if (kt) kt->end(st);
    if (launches) *launches += 5;
}

}  // namespace lc

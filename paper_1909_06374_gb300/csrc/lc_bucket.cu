// lc_bucket.cu -- the rank-order replacement of one E13 iteration (Sec. 2.1
// third step, Sec. 3.2.2: x[perm[r]] = s[r] with perm the stable argsort of
// x_adj) as a sample sort: one bucket pass through HBM and one on-chip pass
// that ranks every element exactly.
//
// Per curve of N = 2^13 .. 2^20 FP32 samples:
//   k_bk_sample   S values of x_adj at a fixed stride (S = 1024 up to 2^17,
//                 4096 above; stored by the inverse transform's last pass,
//                 or gathered here), sorted in registers and shared
//                 memory; every (S/256)-th becomes one of the splitters of 256
//                 buckets (bucket b holds spl[b-1] <= x < spl[b]); a
//                 4096-cell grid over the sample's range with, per cell, the
//                 number of splitters in earlier cells;
//   k_bk_hist     per 2048-element tile: bucket of every element (its cell's
//                 count, plus the splitters of its own cell that do not
//                 exceed it; one byte per element kept for the scatter) and
//                 the tile's bucket counts;
//   k_bk_scan     tile prefixes and bucket bases of the curve, each bucket's
//                 bounds, and groups of consecutive buckets of at most CAP
//                 elements (2048 up to 2^18, N/128 above), in the curve's
//                 own work-item slots;
//   k_bk_scatter  per tile: the elements placed in shared memory in bucket
//                 order (the order inside a bucket is arbitrary), then each
//                 bucket's run written to the tile's slice of the bucket;
//   k_bk_finish   one work item per block, in shared memory: every bucket is
//                 split into two sub-buckets per element by linear
//                 interpolation of the value between the bucket's bounds
//                 (monotone; values beyond the sample's extremes go to the
//                 edge sub-buckets); the elements are counted per sub-bucket
//                 and the counts scanned; an element alone in its sub-bucket
//                 has the sub-bucket's start as rank, the members of a shared
//                 one are placed side by side and ranked among themselves by
//                 (value, position) -- the stable argsort order, whatever
//                 order the scatter left.  rank = group base + rank in the
//                 group; the block writes x[position] = s[rank].  Blocks
//                 are launched for the first glaunch slots of each curve;
//   k_bk_finish_tail one block per curve for any groups beyond them.
// A bucket of more than CAP elements (a spike of equal or nearly equal
// values, or rarely a wide bucket) is one group of its own, sorted by a
// block-level LSD radix sort on (value, position) through global memory
// instead.
//
// HBM bytes per element: 4 (histogram) + 4 + 1 + 8 (scatter, incl. the
// bucket byte) + 8 + 4 + 4 (finish) + 1 (bucket byte written) = 34, against
// 76 for the four 8-bit LSD passes and their histograms.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "lc_internal.h"

namespace lc {

constexpr int kBkBuckets = 256;
constexpr int kBkTileThreads = 256;              // histogram and scatter kernels

// Sample size and finish-group capacity per length.  Up to 2^17: 1024 sample
// values (four per bucket) and groups of at most 2048 elements.  From 2^18
// on: 4096 values (16 per bucket: bucket sizes spread less, 0.07% of buckets
// exceed twice the mean) and groups of twice the mean bucket, N / 128: 2048
// at 2^18, 4096 at 2^19, 8192 at 2^20.
int bucket_samples(uint32_t log2n)
{
    return log2n >= 18 ? 4096 : 1024;
}

int bucket_cap(uint32_t log2n)
{
    return log2n <= 18 ? kBkCap : (kBkCap << (log2n - 18));
}

// Auxiliary area of a class (u32 words): a 64-word header (unused), then per
// curve: splitters (float bits), the curve's min and max (order keys), bucket
// bases (257), the group count, per-bucket parameters (lower bound, elements
// per unit value, base, count: 4 words each), the bucket-search grid (lo,
// cells per unit value) and its table (one byte per cell), the sample of
// x_adj (bucket_samples floats, written by the inverse transform's last
// pass); then the work items of the finish kernel, gmax slots per curve (e0,
// n, first bucket, buckets; curve offset lo, hi, class index of the curve, 0:
// 8 words each; n = 0 in the slots after the curve's groups).
constexpr int kAuxHeader = 64;
constexpr int kAuxSpl = 0;
constexpr int kAuxMin = 256;
constexpr int kAuxMax = 257;
constexpr int kAuxBase = 258;
constexpr int kAuxGcount = kAuxBase + kBkBuckets + 1;   // 515
constexpr int kAuxPar = 516;                            // 16-byte aligned
constexpr int kBkCells = 4096;                          // lookup cells of the bucket search
constexpr int kAuxGrid = kAuxPar + 4 * kBkBuckets;      // lo (float bits), cells per unit value (float bits)
constexpr int kAuxLut = kAuxGrid + 4;                   // kBkCells bytes: splitters in earlier cells
constexpr int kAuxSmp = (kAuxLut + kBkCells / 4 + 3) / 4 * 4;  // the sample's floats

int bucket_curve_words(uint32_t log2n)
{
    return ((kAuxSmp + bucket_samples(log2n)) + 63) / 64 * 64;
}

float* bucket_sample_area(const ClassInfo& k)
{
    return (float*)(k.d_aux + kAuxHeader + kAuxSmp);
}

// Sample i of a curve of N = 2^log2n samples, S = bucket_samples(log2n), is
// x_adj[i N/S + N/(2 S)], the real part of complex element d = i 2^shift +
// 2^(shift-1) with 2^shift = N / (2 S).
uint32_t bucket_sample_shift(uint32_t log2n)
{
    return log2n - 1 - (bucket_samples(log2n) == 4096 ? 12u : 10u);
}

int bucket_gmax(uint32_t log2n)
{
    // greedy groups: any two consecutive ones hold more than the capacity
    return 2 * (int)(((size_t)1 << log2n) / (size_t)bucket_cap(log2n)) + 1;
}

// Finish blocks launched per curve: a little above the 99.9th percentile of
// the number of groups per curve (measured on a model of the splitter
// sample: at 2^16 35 groups on average, 36 at most, of gmax = 65 slots; from
// 2^18 on about 178 of 257), so that few launched blocks find an empty slot.
// A curve with more groups has the rest finished by k_bk_finish_tail.
int bucket_glaunch(uint32_t log2n)
{
    static const int tab[] = {6, 10, 19, 38, 83, 189, 189, 189};  // 2^13 .. 2^20
    const int i = (int)log2n - 13;
    const int g = (i >= 0 && i < 8) ? tab[i] : bucket_gmax(log2n);
    return std::min(g, bucket_gmax(log2n));
}

size_t bucket_aux_words(uint32_t log2n, int ncurves)
{
    return (size_t)kAuxHeader + (size_t)ncurves * bucket_curve_words(log2n) +
           8 * (size_t)ncurves * bucket_gmax(log2n);
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
    int presampled;          // the sample is in the aux area already
    uint32_t* aux;           // [ci][cw]
    uint4* items;            // [2 * (ci gmax + g)]: e0, n, first bucket, buckets; off lo, hi, ci, 0
    uint32_t* hist;          // [ci][tpc][256]
    uint32_t* bid;           // bucket of every element, one byte each (four per word)
    uint32_t* keys;          // bucket order: value bits
    uint32_t* vals;          // bucket order: position | bucket << 24
    uint32_t* keys2;         // ping-pong of the oversize-bucket sort
    uint32_t* vals2;
    const float* s;          // sorted draws
    float* x_out;            // x[position] = s[rank]
    int tpc;
    int gmax;
    int cw;                  // aux words per curve
    int cap;                 // finish-group capacity (elements)
    int glaunch;             // finish blocks launched per curve (<= gmax)
    uint32_t log2n;
};

__device__ __forceinline__ bool bk_active(const BkArgs& a, int c)
{
    return !a.d_iter || (uint32_t)(*a.d_iter) < a.eff_iters[c];
}

// Cell of v on the bucket-search grid: monotone in v, in [0, kBkCells).
__device__ __forceinline__ int grid_cell(float v, float lo, float scale)
{
    return max(0, min(__float2int_rz((v - lo) * scale), kBkCells - 1));  // NaN -> 0
}

// Number of splitters <= v: the bucket of v (spl ascending, 255 entries
// used).  lut[c] = splitters in cells below c, a lower bound of the bucket of
// every value of cell c; the splitters of the value's own cell that do not
// exceed it are counted on top (any splitter of a later cell exceeds it).
__device__ __forceinline__ uint32_t bucket_of(const float* spl, const uint8_t* lut, float lo, float scale, float v)
{
    uint32_t b = lut[grid_cell(v, lo, scale)];
    while (b < kBkBuckets - 1 && v >= spl[b]) ++b;
    return b;
}

// ------------------------------------------------------------------ sample
// Compare-exchange of a bitonic stage: the element with the lower index of the
// pair keeps the smaller value in an ascending block (bit k of its index 0).
__device__ __forceinline__ float bitonic_keep(float mine, float other, bool lower, bool up)
{
    const bool keep_min = lower == up;
    return keep_min ? (other < mine ? other : mine) : (other > mine ? other : mine);
}

// A bitonic stage whose pairs are elements i and i + M of one thread (element
// index 32 (8 warp + i) + lane): M is a compile-time constant so that v stays
// in registers.
template <int M>
__device__ __forceinline__ void bitonic_in_thread(float (&v)[8], int warp, int lane, int k)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((i & M) == 0) {
            const int e = 32 * (8 * warp + i) + lane;
            const float x0 = v[i], x1 = v[i + M];
            const bool up = (e & k) == 0;
            v[i] = bitonic_keep(x0, x1, true, up);
            v[i + M] = bitonic_keep(x1, x0, false, up);
        }
    }
}

// Cell-count index with one pad word per 32 cells, so that a thread reading
// its own 32 consecutive cells meets no bank conflict with its warp.
__device__ __forceinline__ int cell_slot(int c)
{
    return c + (c >> 5);
}

// One block of S / 8 threads per curve (S = 1024 or 4096 sample values).  The
// sample is sorted by a bitonic network held in registers: thread (warp w,
// lane l) keeps element 32 (8 w + i) + l in v[i], i < 8, so the stages with a
// partner distance j < 32 exchange through warp shuffles, those with j = 32,
// 64, 128 stay inside the thread, and only j >= 256 go through shared memory.
template <int S, bool MULTI>
__global__ void __launch_bounds__(S / 8) k_bk_sample(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    constexpr int TH = S / 8;  // 8 elements per thread
    constexpr int PER = 8;
    static_assert(S == 1024 || S == 4096, "register layout of the sample sort");
    const int ci = (int)blk;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float sm[S];
    __shared__ uint32_t cnt[kBkCells + kBkCells / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t* A0 = a.aux + (size_t)ci * a.cw;
    float v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = 32 * (8 * warp + i) + lane;
        if (a.presampled) {
            v[i] = __uint_as_float(A0[kAuxSmp + e]);
        } else {
            const uint32_t stride = (1u << a.log2n) / (uint32_t)S;
            v[i] = a.xadj[a.curves[c].off + (uint64_t)e * stride + stride / 2];
        }
    }
    for (int i = tid; i < kBkCells + kBkCells / 32; i += TH) cnt[i] = 0u;
    // bitonic sort, ascending
    for (int k = 2; k <= S; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < 32) {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int e = 32 * (8 * warp + i) + lane;
                    const float o = __shfl_xor_sync(0xffffffffu, v[i], j);
                    v[i] = bitonic_keep(v[i], o, lower, (e & k) == 0);
                }
            } else if (j < 256) {  // partner: element i ^ (j / 32) of the same thread
                if (j == 32) bitonic_in_thread<1>(v, warp, lane, k);
                else if (j == 64) bitonic_in_thread<2>(v, warp, lane, k);
                else bitonic_in_thread<4>(v, warp, lane, k);
            } else {
#pragma unroll
                for (int i = 0; i < PER; ++i) sm[32 * (8 * warp + i) + lane] = v[i];
                __syncthreads();
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int e = 32 * (8 * warp + i) + lane;
                    v[i] = bitonic_keep(v[i], sm[e ^ j], (e & j) == 0, (e & k) == 0);
                }
                __syncthreads();
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) sm[32 * (8 * warp + i) + lane] = v[i];
    __syncthreads();
    uint32_t* A = a.aux + (size_t)ci * a.cw;
    // splitters; the search grid spans the sample's range
    const float glo = sm[0], ghi = sm[S - 1];
    const float d = ghi - glo;
    const float gscale = d > 0.0f ? (float)kBkCells / d : 0.0f;
    for (int i = tid; i < kBkBuckets; i += TH) {
        if (i < kBkBuckets - 1) {
            const float sv = sm[(S / kBkBuckets) * (i + 1)];
            A[kAuxSpl + i] = __float_as_uint(sv);
            atomicAdd(&cnt[cell_slot(grid_cell(sv, glo, gscale))], 1u);
        } else {
            A[kAuxSpl + i] = 0x7f800000u;  // +inf, never compared
        }
    }
    if (tid == 0) {
        // the sample's extremes bound the first and the last bucket (values
        // beyond them go to those buckets' edge sub-buckets)
        A[kAuxMin] = order_key(glo);
        A[kAuxMax] = order_key(ghi);
        A[kAuxGrid] = __float_as_uint(glo);
        A[kAuxGrid + 1] = __float_as_uint(gscale);
    }
    __syncthreads();
    // lut[c] = splitters in cells below c: exclusive scan of the cell counts
    // (thread tid owns kBkCells / threads consecutive cells)
    {
        constexpr int CPT = kBkCells / TH;  // 32 or 8
        static_assert(CPT % 4 == 0, "whole table words per thread");
        const int c0 = tid * CPT;
        uint32_t run = 0;
#pragma unroll
        for (int q = 0; q < CPT; ++q) run += cnt[cell_slot(c0 + q)];
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __shared__ uint32_t wsum[TH / 32];
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t acc = incl - run;
        for (int w = 0; w < warp; ++w) acc += wsum[w];
        uint32_t* lut = A + kAuxLut;
#pragma unroll
        for (int q = 0; q < CPT; q += 4) {
            uint32_t word = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                word |= min(acc, 255u) << (8 * t);
                acc += cnt[cell_slot(c0 + q + t)];
            }
            lut[(c0 + q) / 4] = word;
        }
    }
}

// ------------------------------------------------------------------ histogram
// TPB tiles per block: bucket counts per tile and the bucket of every element
// (one byte, packed four to a word, for the scatter).
template <int TPB, bool MULTI>
__global__ void __launch_bounds__(kBkTileThreads) k_bk_hist(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    constexpr int V4 = kSortTile / 4 / kBkTileThreads;  // float4 loads per thread and tile
    const int bpc = a.tpc / TPB;
    const int ci = (int)blk / bpc;
    const int t0 = ((int)blk % bpc) * TPB;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float spl[kBkBuckets];
    __shared__ uint32_t lutw[kBkCells / 4];
    __shared__ uint32_t h[TPB][kBkBuckets];
    const int tid = threadIdx.x;
    uint32_t* A = a.aux + (size_t)ci * a.cw;
    spl[tid] = __uint_as_float(A[kAuxSpl + tid]);
    for (int i = tid; i < kBkCells / 4; i += kBkTileThreads) lutw[i] = A[kAuxLut + i];
    const float glo = __uint_as_float(A[kAuxGrid]), gscale = __uint_as_float(A[kAuxGrid + 1]);
    const uint8_t* lut = (const uint8_t*)lutw;
#pragma unroll
    for (int u = 0; u < TPB; ++u) h[u][tid] = 0;
    const uint64_t off = a.curves[c].off;
    const float4* __restrict__ src = (const float4*)(a.xadj + off + (uint64_t)t0 * kSortTile);
    uint32_t* __restrict__ bid = a.bid + off + (uint64_t)t0 * (kSortTile / 4);
    float4 q[TPB * V4];
#pragma unroll
    for (int e = 0; e < TPB * V4; ++e) {
        const int u = e / V4, v = tid + (e % V4) * kBkTileThreads;
        q[e] = src[(size_t)u * (kSortTile / 4) + v];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < TPB * V4; ++e) {
        const int u = e / V4, v = tid + (e % V4) * kBkTileThreads;
        const float vv[4] = {q[e].x, q[e].y, q[e].z, q[e].w};
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t b = bucket_of(spl, lut, glo, gscale, vv[j]);
            atomicAdd(&h[u][b], 1u);
            word |= b << (8 * j);
        }
        bid[(size_t)u * (kSortTile / 4) + v] = word;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPB; ++u) a.hist[((size_t)ci * a.tpc + t0 + u) * kBkBuckets + tid] = h[u][tid];
}

// ------------------------------------------------------------------ scan
// One block (256 threads, thread b = bucket b) per curve.  The curve's groups
// take its gmax work-item slots in order; the slots after them are marked
// empty (n = 0), and so are all of them for a curve that has stopped.
// Groups: the group that starts at bucket s ends before bucket e = the last
// index with base[e] - base[s] <= cap (at least s + 1: a larger bucket is a
// group of its own), found for every s at once by binary search; thread 0
// then follows these links from bucket 0.  Any two consecutive groups hold
// more than cap elements, so a curve has at most gmax = 2 N / cap + 1.
template <bool MULTI>
__global__ void __launch_bounds__(kBkBuckets) k_bk_scan(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    constexpr int kChunk = 32;  // tile counts loaded together
    const int ci = (int)blk;
    const int c = a.cls_curves[ci];
    uint4* items = a.items + 2 * (size_t)ci * a.gmax;
    if (!bk_active(a, c)) {
        for (int g = threadIdx.x; g < a.gmax; g += kBkBuckets) items[2 * g] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    __shared__ uint32_t wsum[kBkBuckets / 32];
    __shared__ uint32_t bs[kBkBuckets + 1];
    __shared__ uint32_t nx[kBkBuckets];
    __shared__ uint32_t gs[kBkBuckets + 1];
    __shared__ uint32_t ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* A = a.aux + (size_t)ci * a.cw;
    // the bucket's bounds (read before the counts, so both loads overlap)
    const float lo = tid == 0 ? key_value(A[kAuxMin]) : __uint_as_float(A[kAuxSpl + tid - 1]);
    const float hi = tid == kBkBuckets - 1 ? key_value(A[kAuxMax]) : __uint_as_float(A[kAuxSpl + tid]);
    // bucket tid's count in every tile, replaced by the tile's prefix
    uint32_t* h = a.hist + (size_t)ci * a.tpc * kBkBuckets + tid;
    uint32_t run = 0;
    for (int t0 = 0; t0 < a.tpc; t0 += kChunk) {
        uint32_t v[kChunk];
        // all of the chunk's loads are issued before any store (the stores
        // overwrite the same words, so the compiler would otherwise pair them)
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            v[u] = 0u;
            if (t0 + u < a.tpc)
                asm volatile("ld.global.u32 %0, [%1];" : "=r"(v[u]) : "l"(h + (size_t)(t0 + u) * kBkBuckets) : "memory");
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
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
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    const uint32_t base = woff + incl - run;
    A[kAuxBase + tid] = base;
    bs[tid] = base;
    if (tid == kBkBuckets - 1) {
        A[kAuxBase + kBkBuckets] = base + run;
        bs[kBkBuckets] = base + run;
    }
    {
        // sub-buckets per unit value (spread linearly over [lo, hi])
        const float d = hi - lo;
        const float sc = (d > 0.0f && run > 0u) ? (float)run / d : 0.0f;
        ((uint4*)(A + kAuxPar))[tid] = make_uint4(__float_as_uint(lo), __float_as_uint(sc), base, run);
    }
    __syncthreads();
    {
        const uint32_t target = base + (uint32_t)a.cap;
        int l = tid + 1, r = kBkBuckets;  // last e in [tid + 1, 256] with bs[e] <= target, else tid + 1
        while (l < r) {
            const int mid = (l + r + 1) >> 1;
            if (bs[mid] <= target) l = mid;
            else r = mid - 1;
        }
        nx[tid] = (uint32_t)l;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t g = 0, b = 0;
        while (b < (uint32_t)kBkBuckets) {
            gs[g++] = b;
            b = nx[b];
        }
        gs[g] = kBkBuckets;
        ng = g;
        A[kAuxGcount] = g;
    }
    __syncthreads();
    const uint64_t off = a.curves[c].off;
    for (int g = tid; g < a.gmax; g += kBkBuckets) {
        if (g < (int)ng) {
            const uint32_t b0 = gs[g], b1 = gs[g + 1];
            items[2 * g] = make_uint4(bs[b0], bs[b1] - bs[b0], b0, b1 - b0);
            items[2 * g + 1] = make_uint4((uint32_t)off, (uint32_t)(off >> 32), (uint32_t)ci, 0u);
        } else {
            items[2 * g] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// ------------------------------------------------------------------ scatter
// One tile per block: its elements are placed in shared memory in bucket
// order (slot atomics: the order inside a bucket is arbitrary), then each
// bucket's run is written to the tile's slice of the bucket with coalesced
// stores.
template <bool MULTI>
__global__ void __launch_bounds__(kBkTileThreads) k_bk_scatter(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    constexpr int V4 = kSortTile / 4 / kBkTileThreads;
    const int ci = (int)blk / a.tpc;
    const int t = (int)blk % a.tpc;
    const int c = a.cls_curves[ci];
    if (!bk_active(a, c)) return;
    __shared__ float stk[kSortTile];
    __shared__ uint32_t stv[kSortTile];
    __shared__ uint32_t cur[kBkBuckets];
    __shared__ uint32_t gb[kBkBuckets];
    __shared__ uint32_t wsum[kBkTileThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t* A = a.aux + (size_t)ci * a.cw;
    const uint64_t off = a.curves[c].off;
    const uint32_t e0 = (uint32_t)t * kSortTile;
    const float4* __restrict__ src = (const float4*)(a.xadj + off + e0);
    const uint32_t* __restrict__ bid = a.bid + off + e0 / 4;
    float4 q[V4];
    uint32_t bw[V4];
#pragma unroll
    for (int e = 0; e < V4; ++e) {
        q[e] = src[tid + e * kBkTileThreads];
        bw[e] = bid[tid + e * kBkTileThreads];
    }
    {
        // the tile's count of bucket tid from the scanned tile prefixes
        const uint32_t* hp = a.hist + ((size_t)ci * a.tpc + t) * kBkBuckets + tid;
        const uint32_t pt = hp[0];
        const uint32_t pn = t + 1 < a.tpc ? hp[kBkBuckets] : A[kAuxBase + tid + 1] - A[kAuxBase + tid];
        const uint32_t n = pn - pt;
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t woff = 0;
        for (int w = 0; w < warp; ++w) woff += wsum[w];
        const uint32_t ls = woff + incl - n;   // the tile's first slot of bucket tid
        cur[tid] = ls;
        gb[tid] = A[kAuxBase + tid] + pt - ls;  // output index of slot i of bucket tid: gb + i
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < V4; ++e) {
        const float vv[4] = {q[e].x, q[e].y, q[e].z, q[e].w};
        const uint32_t i0 = e0 + 4u * (uint32_t)(tid + e * kBkTileThreads);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t b = (bw[e] >> (8 * j)) & 255u;
            const uint32_t slot = atomicAdd(&cur[b], 1u);
            stk[slot] = vv[j];
            stv[slot] = (i0 + (uint32_t)j) | (b << 24);
        }
    }
    __syncthreads();
    uint32_t* __restrict__ kd = a.keys + off;
    uint32_t* __restrict__ vd = a.vals + off;
#pragma unroll
    for (int e = 0; e < kSortTile / kBkTileThreads; ++e) {
        const int i = tid + e * kBkTileThreads;
        const uint32_t v = stv[i];
        const uint32_t dst = gb[v >> 24] + (uint32_t)i;
        kd[dst] = __float_as_uint(stk[i]);
        vd[dst] = v;
    }
}

// ------------------------------------------------------------------ finish
// Block-wide exclusive scan of v (TH threads).
template <int TH>
__device__ __forceinline__ uint32_t bk_block_scan(uint32_t v, uint32_t* wsum)
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
    uint32_t woff = 0;
#pragma unroll
    for (int w = 0; w < TH / 32; ++w) woff += w < warp ? wsum[w] : 0u;
    __syncthreads();
    return woff + incl - v;
}

// One stable LSD pass of the block over n (key, val) pairs in global memory,
// by the byte `shift` of the position (val, bits 0..23) when !KEYB, else of
// the value's order key.  Returns false (nothing moved) when every element
// has the same digit.
template <bool KEYB, int TH>
__device__ bool bk_block_pass(const uint32_t* __restrict__ ik, const uint32_t* __restrict__ iv,
                              uint32_t* __restrict__ ok, uint32_t* __restrict__ ov, int n, int shift,
                              uint32_t* hist, uint32_t (*wc)[256], uint32_t* wsum)
{
    constexpr int W = TH / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto digit = [&](uint32_t k, uint32_t v) -> uint32_t {
        return KEYB ? (order_key(__uint_as_float(k)) >> shift) & 255u : ((v & 0xffffffu) >> shift) & 255u;
    };
    static_assert(TH >= 256, "one thread per digit");
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += TH) atomicAdd(&hist[digit(ik[i], iv[i])], 1u);
    __syncthreads();
    if (__syncthreads_or(tid < 256 && hist[tid] == (uint32_t)n)) return false;
    uint32_t base = bk_block_scan<TH>(tid < 256 ? hist[tid] : 0u, wsum);  // digit tid's first output index
    const uint32_t lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < n; c0 += TH) {
        for (int q = tid; q < W * 256; q += TH) (&wc[0][0])[q] = 0;
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
template <int TH>
__device__ void bk_oversize(const BkArgs& a, uint64_t off, uint32_t e0, int n, uint32_t* smem_u32)
{
    uint32_t* hist = smem_u32;
    uint32_t(*wc)[256] = (uint32_t(*)[256])(smem_u32 + 256);
    uint32_t* wsum = smem_u32 + 256 + (TH / 32) * 256;
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
        const bool moved = keyb ? bk_block_pass<true, TH>(ik, iv, ok, ov, n, shift, hist, wc, wsum)
                                : bk_block_pass<false, TH>(ik, iv, ok, ov, n, shift, hist, wc, wsum);
        if (moved) in0 = !in0;
    }
    const uint32_t* vf = in0 ? v0 : v1;
    const float* __restrict__ s = a.s + off + e0;
    float* __restrict__ x = a.x_out + off;
    for (int r = threadIdx.x; r < n; r += TH) x[vf[r] & 0xffffffu] = s[r];
}

// Sub-buckets per element of a bucket (linear interpolation of the value
// between the bucket's bounds): fewer elements share one, so fewer need the
// comparison step; their counters are 16 bits wide (two to a word), so two
// per element cost no more shared memory or scan steps than one 32-bit
// counter per element.
constexpr int kBkSubPer = 2;

// Finish kernel of groups of at most CAP elements: 512 threads of four
// elements (four blocks per SM) at CAP = 2048, 1024 threads of four (two
// blocks per SM) at 4096, 1024 threads of eight (one block per SM) at 8192.
// Shared memory (u32 words): the 64-bit keys (order key of the value << 32 |
// position) of the elements that share a sub-bucket, at their sub-bucket's
// start + arrival index; sub-bucket counts, then starts (nsub + 1, 16 bits
// each, two to a word); per-bucket parameters; scan partials.
template <int CAP>
struct FinLayout {
    static constexpr int THREADS = CAP == 2048 ? 512 : 1024;
    static constexpr int PER = CAP / THREADS;            // elements per thread
    static constexpr int MINB = CAP == 2048 ? 4 : (CAP == 4096 ? 2 : 1);
    static constexpr int NSUB = kBkSubPer * CAP;
    static constexpr int KK = 0;                         // CAP u64
    static constexpr int ST = 2 * CAP;                   // NSUB / 2 + 1 words (+3 pad)
    static constexpr int PAR = ST + NSUB / 2 + 4;        // float2 lo/scale, uint2 first/count: 4 x 256
    static constexpr int WS = PAR + 4 * kBkBuckets;      // THREADS / 32
    static constexpr int WORDS = WS + 32;
    static constexpr size_t SMEM = (size_t)WORDS * 4;
    static_assert(WORDS >= 256 + (THREADS / 32) * 256 + 16, "oversize sort scratch");
    static_assert(THREADS / 32 <= 32, "scan partials");
    static_assert(NSUB <= 65536 && CAP <= 65535, "sub-bucket, arrival index and starts in 16 bits");
};

// One work-item slot per block (gmax slots per curve); a block whose slot is
// empty returns at once.
// Ranks the elements of work item `item` (a group of buckets of one curve)
// and writes x[position] = s[rank]; false when the item is empty.
template <int CAP>
__device__ __forceinline__ bool bk_finish_item(const BkArgs& a, uint32_t item, uint32_t* bsm)
{
    using L = FinLayout<CAP>;
    constexpr int TH = L::THREADS, PER = L::PER;
    constexpr uint32_t kPosMask = (1u << 24) - 1u;
    const uint4 d0 = a.items[2 * item];
    const uint4 d1 = a.items[2 * item + 1];
    const uint32_t e0 = d0.x, b0 = d0.z;
    const int n = (int)d0.y, nb = (int)d0.w;
    if (n == 0) return false;
    const uint64_t off = (uint64_t)d1.x | ((uint64_t)d1.y << 32);
    const uint32_t* A = a.aux + (size_t)d1.z * a.cw;
    if (n > CAP) {  // one bucket of nearly equal values
        bk_oversize<TH>(a, off, e0, n, bsm);
        return true;
    }
    const int ns = kBkSubPer * n;  // sub-buckets of the group
    unsigned long long* kk = (unsigned long long*)(bsm + L::KK);
    uint32_t* st = bsm + L::ST;
    float2* plo = (float2*)(bsm + L::PAR);                 // (lower bound, sub-buckets per unit)
    uint2* pof = (uint2*)(bsm + L::PAR + 2 * kBkBuckets);  // (first sub-bucket, sub-buckets)
    uint32_t* wsum = bsm + L::WS;
    const int tid = threadIdx.x;
    const uint32_t* __restrict__ kin = a.keys + off + e0;
    const uint32_t* __restrict__ vin = a.vals + off + e0;
    float key[PER];
    uint32_t pos[PER], sub[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = tid + j * TH;
        if (p < n) {
            key[j] = __uint_as_float(kin[p]);
            pos[j] = vin[p];
        }
    }
    static_assert(TH >= kBkBuckets, "one thread per bucket of a group");
    if (tid < nb) {
        const uint4 P = ((const uint4*)(A + kAuxPar))[b0 + (uint32_t)tid];
        // P.y: elements per unit value; kBkSubPer sub-buckets per element
        plo[tid] = make_float2(__uint_as_float(P.x), (float)kBkSubPer * __uint_as_float(P.y));
        pof[tid] = make_uint2((uint32_t)kBkSubPer * (P.z - e0), (uint32_t)kBkSubPer * P.w);
    }
    const int nw = ns / 2;  // words of the 16-bit counters
    for (int i = tid; i <= nw; i += TH) st[i] = 0u;
    __syncthreads();
    // count: the sub-bucket of every element (kBkSubPer per element of its
    // bucket, by linear interpolation between the bucket's bounds: monotone in
    // the value) and its arrival index in it
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = tid + j * TH;
        if (p < n) {
            const uint32_t bl = min((pos[j] >> 24) - b0, (uint32_t)nb - 1u);
            pos[j] &= kPosMask;
            const float2 ls = plo[bl];
            const uint2 of = pof[bl];
            int q = __float2int_rz((key[j] - ls.x) * ls.y);  // NaN -> 0
            q = max(0, min(q, (int)of.y - 1));
            const uint32_t u = of.x + (uint32_t)q;
            const uint32_t sh = (u & 1u) << 4;  // 16-bit counter u: half u & 1 of word u / 2
            const uint32_t old = (atomicAdd(&st[u >> 1], 1u << sh) >> sh) & 0xffffu;
            sub[j] = u | (old << 16);
        }
    }
    __syncthreads();
    // exclusive scan of the ns 16-bit sub-bucket counts in place (thread tid
    // owns the consecutive words from kSc tid); st16[ns] = n
    uint16_t* st16 = (uint16_t*)st;
    {
        constexpr int kSc = L::NSUB / 2 / TH;
        static_assert(kSc % 4 == 0, "16-byte loads");
        const int q0 = tid * kSc;
        // the counts are read twice (sum, then prefixes) to keep them out of
        // registers while the elements' state is live
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < kSc; j += 4) {
            if (q0 + j < nw) {
                const uint4 v = *(const uint4*)(st + q0 + j);  // words to nw + 3: zeroed or counted
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (q0 + j + t < nw) sum += (w[t] & 0xffffu) + (w[t] >> 16);
            }
        }
        uint32_t run = bk_block_scan<TH>(sum, wsum);
#pragma unroll
        for (int j = 0; j < kSc; j += 4) {
            if (q0 + j < nw) {
                const uint4 v = *(const uint4*)(st + q0 + j);
                uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t lo = run;
                    if (q0 + j + t < nw) run += w[t] & 0xffffu;
                    const uint32_t hi = run;
                    if (q0 + j + t < nw) run += w[t] >> 16;
                    w[t] = lo | (hi << 16);
                }
                *(uint4*)(st + q0 + j) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
    __syncthreads();
    if (tid == 0) st16[ns] = (uint16_t)n;
    __syncthreads();
    // an element alone in its sub-bucket has rank = the sub-bucket's start;
    // the members of a shared sub-bucket are placed at start + arrival index
    // and ranked below.  rk[j] = the start; sub[j] = members | arrival << 16
    uint32_t rk[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = tid + j * TH;
        if (p < n) {
            const uint32_t u = sub[j] & 0xffffu, old = sub[j] >> 16;
            const uint32_t s0 = st16[u];
            const uint32_t c = st16[u + 1] - s0;
            rk[j] = s0;
            if (c > 1u) kk[s0 + old] = ((unsigned long long)order_key(key[j]) << 32) | pos[j];
            sub[j] = c | (old << 16);
        }
    }
    __syncthreads();
    const float* __restrict__ s = a.s + off + e0;
    float* __restrict__ x = a.x_out + off;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = tid + j * TH;
        if (p < n) {
            uint32_t r = rk[j];
            const uint32_t c = sub[j] & 0xffffu;
            if (c > 1u) {
                // rank among the members by (value, position): one 64-bit
                // comparison per member (order keys of equal values are
                // equal, positions break the tie)
                const unsigned long long K = ((unsigned long long)order_key(key[j]) << 32) | pos[j];
                const uint32_t s0 = r;
                for (uint32_t m = s0; m < s0 + c; ++m) r += kk[m] < K ? 1u : 0u;
            }
            x[pos[j]] = s[r];
        }
    }
    return true;
}

// One block per launched work-item slot: glaunch slots per curve, enough for
// the groups of almost every curve (a curve's groups fill its first slots, any
// later slot is empty).
template <int CAP, bool MULTI>
__global__ void __launch_bounds__(FinLayout<CAP>::THREADS, FinLayout<CAP>::MINB)
    k_bk_finish(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    extern __shared__ __align__(16) uint32_t bsm[];
    const uint32_t gl = (uint32_t)a.glaunch;
    const uint32_t ci = blk / gl, g = blk - ci * gl;
    bk_finish_item<CAP>(a, ci * (uint32_t)a.gmax + g, bsm);
}

// The groups of a curve beyond its glaunch launched slots, if any: one block
// per curve, one group after the other (almost always none).  The loop runs
// to the curve's group count, not to the first empty item: a group of empty
// buckets (before an oversize bucket) has no elements but later groups do.
template <int CAP, bool MULTI>
__global__ void __launch_bounds__(FinLayout<CAP>::THREADS, FinLayout<CAP>::MINB)
    k_bk_finish_tail(const __grid_constant__ LaunchSet<BkArgs> set)
{
    uint32_t blk;
    const BkArgs& a = set.pick<MULTI>(blk);
    extern __shared__ __align__(16) uint32_t bsm[];
    const uint32_t gm = (uint32_t)a.gmax;
    const uint32_t ng = min(a.aux[(size_t)blk * a.cw + kAuxGcount], gm);
    for (uint32_t h = (uint32_t)a.glaunch; h < ng; ++h) {
        if (bk_finish_item<CAP>(a, blk * gm + h, bsm)) __syncthreads();  // the next group reuses the shared memory
    }
}

template <int CAP>
static cudaError_t finish_attrs()
{
    const int smem = (int)FinLayout<CAP>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_bk_finish<CAP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bk_finish<CAP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bk_finish_tail<CAP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bk_finish_tail<CAP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t bucket_kernel_attributes()
{
    cudaError_t e = finish_attrs<2048>();
    if (e == cudaSuccess) e = finish_attrs<4096>();
    if (e == cudaSuccess) e = finish_attrs<8192>();
    return e;
}

template <int S>
static int launch_sample_sets(const std::vector<BkArgs>& args, const std::vector<uint32_t>& blocks, cudaStream_t st)
{
    return for_launch_sets(args, blocks, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_sample<S, true><<<g, S / 8, 0, st>>>(s);
        else k_bk_sample<S, false><<<g, S / 8, 0, st>>>(s);
    });
}

// The finish launches of one group capacity, then (for the classes that
// launch fewer blocks per curve than they have slots) the tail launches.
template <int CAP>
static int launch_finish_sets(const std::vector<BkArgs>& args, const std::vector<uint32_t>& blocks, cudaStream_t st)
{
    using L = FinLayout<CAP>;
    int n = for_launch_sets(args, blocks, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_finish<CAP, true><<<g, L::THREADS, L::SMEM, st>>>(s);
        else k_bk_finish<CAP, false><<<g, L::THREADS, L::SMEM, st>>>(s);
    });
    std::vector<BkArgs> tail;
    std::vector<uint32_t> tb;
    for (size_t i = 0; i < args.size(); ++i) {
        if (args[i].glaunch >= args[i].gmax) continue;
        tail.push_back(args[i]);
        tb.push_back(blocks[i] / (uint32_t)args[i].glaunch);  // one block per curve
    }
    n += for_launch_sets(tail, tb, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_finish_tail<CAP, true><<<g, L::THREADS, L::SMEM, st>>>(s);
        else k_bk_finish_tail<CAP, false><<<g, L::THREADS, L::SMEM, st>>>(s);
    });
    return n;
}

template <int TPB>
static int launch_hist_sets(const std::vector<BkArgs>& args, const std::vector<uint32_t>& blocks, cudaStream_t st)
{
    return for_launch_sets(args, blocks, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_hist<TPB, true><<<g, kBkTileThreads, 0, st>>>(s);
        else k_bk_hist<TPB, false><<<g, kBkTileThreads, 0, st>>>(s);
    });
}

void launch_bucket_argsort(const Plan& p, const std::vector<const ClassInfo*>& ks,
                           const std::vector<const void*>& srcs, void* x_out, bool gated, bool presampled,
                           cudaStream_t st, uint64_t* launches, KernelTimes* kt)
{
    const size_t nk = ks.size();
    std::vector<BkArgs> args(nk);
    std::vector<uint32_t> b_curve(nk), b_tile(nk), b_item(nk);
    // histogram blocks: two tiles per block (32 registers, eight blocks per
    // SM) where the curve has them
    std::vector<BkArgs> h1, h2;
    std::vector<uint32_t> hb1, hb2;
    for (size_t i = 0; i < nk; ++i) {
        const ClassInfo& k = *ks[i];
        BkArgs& a = args[i];
        a = BkArgs{};
        // only the tile path's inverse transform (log2 N >= 13) writes the sample
        a.presampled = (presampled && k.log2n - 1 >= 12) ? 1 : 0;
        a.cls_curves = k.d_curves;
        a.curves = p.d_curves;
        a.eff_iters = p.d_eff_iters;
        a.d_iter = gated ? p.d_iter : nullptr;
        a.xadj = (const float*)srcs[i];
        a.aux = k.d_aux + kAuxHeader;
        a.items = (uint4*)(k.d_aux + kAuxHeader + (size_t)k.ncurves * bucket_curve_words(k.log2n));
        a.hist = p.d_hist + k.hist_off;
        a.bid = p.d_valsB;  // free until the finish: the bucket bytes of curve c at word off_c
        a.keys = (uint32_t*)p.d_keysA;
        a.vals = p.d_valsA;
        a.keys2 = (uint32_t*)p.d_f;
        a.vals2 = p.d_valsB;
        a.s = (const float*)p.d_s;
        a.x_out = (float*)(x_out ? x_out : p.d_x);
        a.tpc = k.tiles_per_curve;
        a.gmax = bucket_gmax(k.log2n);
        a.cw = bucket_curve_words(k.log2n);
        a.cap = bucket_cap(k.log2n);
        a.glaunch = bucket_glaunch(k.log2n);
        a.log2n = k.log2n;
        b_curve[i] = (uint32_t)k.ncurves;
        b_tile[i] = (uint32_t)(k.ncurves * a.tpc);
        b_item[i] = (uint32_t)(k.ncurves * a.glaunch);
        if (a.tpc >= 2) {
            h2.push_back(a);
            hb2.push_back((uint32_t)(k.ncurves * (a.tpc / 2)));
        } else {
            h1.push_back(a);
            hb1.push_back((uint32_t)(k.ncurves * a.tpc));
        }
    }
    int n = 0;
    if (kt) kt->begin(kGroupSortHistScan, st);
    {
        // one launch per sample size
        std::vector<BkArgs> s1, s4;
        std::vector<uint32_t> b1, b4;
        for (size_t i = 0; i < nk; ++i) {
            (bucket_samples(args[i].log2n) == 4096 ? s4 : s1).push_back(args[i]);
            (bucket_samples(args[i].log2n) == 4096 ? b4 : b1).push_back(b_curve[i]);
        }
        n += launch_sample_sets<1024>(s1, b1, st);
        n += launch_sample_sets<4096>(s4, b4, st);
    }
    n += launch_hist_sets<2>(h2, hb2, st);
    n += launch_hist_sets<1>(h1, hb1, st);
    n += for_launch_sets(args, b_curve, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_scan<true><<<g, kBkBuckets, 0, st>>>(s);
        else k_bk_scan<false><<<g, kBkBuckets, 0, st>>>(s);
    });
    if (kt) kt->end(st);
    if (kt) kt->begin(kGroupSortScatter, st);
    n += for_launch_sets(args, b_tile, [&](const LaunchSet<BkArgs>& s, uint32_t g, bool multi) {
        if (multi) k_bk_scatter<true><<<g, kBkTileThreads, 0, st>>>(s);
        else k_bk_scatter<false><<<g, kBkTileThreads, 0, st>>>(s);
    });
    {
        // one launch per finish capacity
        std::vector<BkArgs> f[3];
        std::vector<uint32_t> fb[3];
        for (size_t i = 0; i < nk; ++i) {
            const int q = args[i].cap == 2048 ? 0 : (args[i].cap == 4096 ? 1 : 2);
            f[q].push_back(args[i]);
            fb[q].push_back(b_item[i]);
        }
        n += launch_finish_sets<2048>(f[0], fb[0], st);
        n += launch_finish_sets<4096>(f[1], fb[1], st);
        n += launch_finish_sets<8192>(f[2], fb[2], st);
    }
    if (kt) kt->end(st);
    if (launches) *launches += (uint64_t)n;
}

void launch_bucket_argsort(const Plan& p, const ClassInfo& k, const void* src, void* x_out, bool gated,
                           bool presampled, cudaStream_t st, uint64_t* launches, KernelTimes* kt)
{
    launch_bucket_argsort(p, std::vector<const ClassInfo*>{&k}, std::vector<const void*>{src}, x_out, gated,
                          presampled, st, launches, kt);
}

}  // namespace lc

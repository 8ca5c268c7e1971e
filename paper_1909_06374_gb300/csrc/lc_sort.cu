// lc_sort.cu -- segmented, stable LSD radix sort of each curve's values with the
// rank-order replacement of the E13 iteration fused into its last pass
// (Sec. 3.2.2: the values are fixed, only their order changes).
//
// Keys are the order-preserving unsigned images of the values (8-bit digits,
// 4 passes for float, 8 for double); the payload is the position k in the
// curve.  Each pass: per-tile digit histograms, a scan (one block per curve
// of at most 32 tiles; tiles in chunks, then chunks, above) giving every
// (tile, digit) its output base, and a stable scatter that ranks the tile in
// shared memory (ballot/match multisplit + per-warp counts) and writes each
// digit's run with coalesced stores.  The last pass of an argsort writes
// x[k] = s[rank] directly instead of the sorted pairs.
#include <algorithm>

#include "lc_internal.h"

namespace lc {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

struct SortArgs {
    const int* cls_curves;
    const CurveDev* curves;
    const uint32_t* eff_iters;
    const int* d_iter;
    const void* src;       // first pass: the values (T)
    const void* keys_in;
    const uint32_t* vals_in;
    void* keys_out;
    uint32_t* vals_out;
    uint32_t* hist;        // [ncurves][tpc][256]
    uint32_t* cbase;       // [ncurves][nchunks][256]
    void* x_out;           // argsort scatter target
    const void* s_in;      // sorted draws
    void* s_out;           // key sort target
    int ncurves;
    int tpc;
    int nchunks;
    int tile_len;
    int shift;
};

__device__ __forceinline__ bool curve_active(const SortArgs& a, int c)
{
    return !a.d_iter || (uint32_t)(*a.d_iter) < a.eff_iters[c];
}

// Key bits of a value stored as T, reinterpreted from the key word.
__device__ __forceinline__ float value_bits(uint32_t b) { return __uint_as_float(b); }
__device__ __forceinline__ double value_bits(unsigned long long b) { return __longlong_as_double((long long)b); }

// Exclusive scan of v over the 256 threads of a block (all threads call it).
__device__ __forceinline__ uint32_t block_exclusive_scan256(uint32_t v, uint32_t* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (int q = 0; q < w; ++q) woff += wsum[q];
    return woff + incl - v;
}

// Curve ci of at most kScanChunk tiles: tile histograms -> exclusive tile
// prefixes in place (digit threadIdx.x), digit bases -> cbase.
__device__ __forceinline__ void scan_curve(const SortArgs& a, int ci, uint32_t* wsum)
{
    const int tid = threadIdx.x;
    uint32_t* hrow = a.hist + (size_t)ci * a.tpc * 256;
    uint32_t v[kScanChunk];
#pragma unroll
    for (int u = 0; u < kScanChunk; ++u) v[u] = u < a.tpc ? __ldcg(&hrow[(size_t)u * 256 + tid]) : 0u;
    uint32_t run = 0;
#pragma unroll
    for (int u = 0; u < kScanChunk; ++u) {
        if (u < a.tpc) hrow[(size_t)u * 256 + tid] = run;
        run += v[u];
    }
    a.cbase[(size_t)ci * 256 + tid] = block_exclusive_scan256(run, wsum);
}

// Per-tile 8-bit digit histograms of TPB consecutive tiles of one curve per
// block: 16-byte loads, all of a thread's loads in flight before the
// counting, per-warp counters.
template <typename T, bool FIRST, int TPB, bool MULTI>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const __grid_constant__ LaunchSet<SortArgs> set)
{
    uint32_t blk;
    const SortArgs& a = set.pick<MULTI>(blk);
    using K = typename key_of<T>::type;
    constexpr int EPV = 16 / (int)sizeof(K);                  // keys per 16-byte load
    constexpr int VPT = kSortTile / EPV / kSortThreads;       // loads per thread and full tile
    const int bpc = a.tpc / TPB;                              // blocks per curve
    const int ci = (int)blk / bpc;
    const int t0 = ((int)blk % bpc) * TPB;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    __shared__ uint32_t h[TPB][kSortWarps][256];
    const int tid = threadIdx.x, warp = tid >> 5;
#pragma unroll
    for (int u = 0; u < TPB; ++u)
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) h[u][w][tid] = 0;
    const uint64_t base = a.curves[c].off + (uint64_t)t0 * a.tile_len;
    const uint4* __restrict__ src = (const uint4*)((const K*)(FIRST ? a.src : a.keys_in) + base);
    const int nvec = a.tile_len / EPV;                        // per tile
    uint4 q[TPB * VPT];
#pragma unroll
    for (int e = 0; e < TPB * VPT; ++e) {
        const int u = e / VPT, v = tid + (e % VPT) * kSortThreads;
        if (v < nvec) q[e] = src[(size_t)u * nvec + v];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < TPB * VPT; ++e) {
        const int u = e / VPT;
        if (tid + (e % VPT) * kSortThreads < nvec) {
            const K* kk = (const K*)&q[e];
#pragma unroll
            for (int j = 0; j < EPV; ++j) {
                const K key = FIRST ? order_key(value_bits(kk[j])) : kk[j];
                atomicAdd(&h[u][warp][(uint32_t)(key >> a.shift) & 255u], 1u);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPB; ++u) {
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) cnt += h[u][w][tid];
        a.hist[((size_t)ci * a.tpc + t0 + u) * 256 + tid] = cnt;
    }
}

// One block per curve of at most kScanChunk tiles: the histograms become tile
// prefixes and the digit bases go to cbase (k_sort_scan_tiles and
// k_sort_scan_chunks in one launch).
template <bool MULTI>
__global__ void __launch_bounds__(256) k_sort_scan_curve(const __grid_constant__ LaunchSet<SortArgs> set)
{
    uint32_t blk;
    const SortArgs& a = set.pick<MULTI>(blk);
    const int ci = (int)blk;
    if (!curve_active(a, a.cls_curves[ci])) return;
    __shared__ uint32_t wsum[kSortWarps];
    scan_curve(a, ci, wsum);
}

// Exclusive prefix of every digit over the tiles of one chunk (in place) and
// the chunk totals.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_sort_scan_tiles(const __grid_constant__ LaunchSet<SortArgs> set)
{
    uint32_t blk;
    const SortArgs& a = set.pick<MULTI>(blk);
    const int ci = (int)blk / a.nchunks;
    const int ch = (int)blk % a.nchunks;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    const int d = threadIdx.x;
    const int t0 = ch * kScanChunk;
    const int nt = min(a.tpc, t0 + kScanChunk) - t0;
    uint32_t* h = a.hist + ((size_t)ci * a.tpc + t0) * 256 + d;
    uint32_t v[kScanChunk];  // all loads issued before the prefix (independent)
#pragma unroll
    for (int t = 0; t < kScanChunk; ++t) v[t] = t < nt ? h[(size_t)t * 256] : 0u;
    uint32_t run = 0;
#pragma unroll
    for (int t = 0; t < kScanChunk; ++t) {
        if (t < nt) h[(size_t)t * 256] = run;
        run += v[t];
    }
    a.cbase[((size_t)ci * a.nchunks + ch) * 256 + d] = run;
}

// Chunk prefixes, digit totals and the digit bases of one curve.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_sort_scan_chunks(const __grid_constant__ LaunchSet<SortArgs> set)
{
    uint32_t blk;
    const SortArgs& a = set.pick<MULTI>(blk);
    const int ci = (int)blk;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    const int d = threadIdx.x;
    uint32_t* cb = a.cbase + (size_t)ci * a.nchunks * 256 + d;
    uint32_t run = 0;
    for (int ch = 0; ch < a.nchunks; ++ch) {
        const uint32_t v = cb[(size_t)ch * 256];
        cb[(size_t)ch * 256] = run;
        run += v;
    }
    // exclusive scan of the digit totals across the block
    __shared__ uint32_t wsum[8];
    const int lane = d & 31, w = d >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (int q = 0; q < w; ++q) woff += wsum[q];
    const uint32_t digit_base = woff + incl - run;
    for (int ch = 0; ch < a.nchunks; ++ch) cb[(size_t)ch * 256] += digit_base;
}

// Lanes of the warp whose 8-bit digit equals this lane's: eight ballots.
__device__ __forceinline__ uint32_t peers8(uint32_t d)
{
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

constexpr int kSlots = kSortTile / kSortThreads;  // elements per thread of a full tile

// Stable scatter of one tile: the tile's elements are ranked in shared memory
// (warp w owns elements [w T/8, (w+1) T/8), lane-striped; ballot/match
// multisplit, per-warp digit counts, one block scan).  MODE 0: the tile is
// placed digit-sorted in shared memory and each digit's run written out with
// coalesced stores of (key, position) pairs, digit d's run starting at gb[d]
// within the curve.  kSortKeysToValues: the same with s[rank] = value.
// kSortArgsortScatter (the last pass of an argsort): every element's rank in
// the curve is gb[d] + (count of d in earlier warps) + (rank in its warp), and
// the element writes x[position] = s[rank] straight from registers (the
// stores are scattered anyway), with no shared-memory placement.
// src_t / src_k / src_v point at the tile's first value / key / position.
// FULL: a tile of kSortTile elements (no bounds tests).  THREADS >= 256 (one
// thread per digit in the per-digit steps).  Expects wcnt zeroed and gb set
// (after a block barrier).  Ends with a block barrier.
template <typename T, bool FIRST, int MODE, bool FULL, int THREADS = kSortThreads>
__device__ __forceinline__ void sort_tile(const SortArgs& a, const T* __restrict__ src_t,
                                          const typename key_of<T>::type* __restrict__ src_k,
                                          const uint32_t* __restrict__ src_v, void* kout, uint32_t* vout, int shift,
                                          uint64_t off, uint32_t e0, int tl, typename key_of<T>::type* sk,
                                          uint32_t* sv, uint32_t (*wcnt)[256], uint32_t* ldstart, uint32_t* gb,
                                          uint32_t* wsum)
{
    using K = typename key_of<T>::type;
    constexpr int WARPS = THREADS / 32;
    constexpr int SLOTS = kSortTile / THREADS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (FULL) tl = kSortTile;
    const int EW = (tl + WARPS - 1) / WARPS;  // elements per warp
    const uint32_t lt = (1u << lane) - 1u;
    K key[SLOTS];
    uint32_t val[SLOTS], rk[SLOTS];
    // ranking in two phases: every slot's load and peer mask first (independent
    // chains that overlap), then the short chain of per-warp digit counters;
    // every second slot takes its mask from the match instruction, the others
    // from eight ballots on the ALU pipe (measured on the 4096 x 2^16 batch:
    // match on none 6.04 ms of scatter per iteration, every 4th 5.62, every
    // 3rd 5.59, every 2nd 5.53)
    uint32_t info[SLOTS];  // digit | below << 8 | count << 16; 0xffffffff: empty slot
#pragma unroll
    for (int e = 0; e < SLOTS; ++e) {
        const int j = e * 32 + lane;              // index within the warp's elements
        const int el = warp * EW + j;             // index within the tile
        const bool valid = FULL || (j < EW && el < tl);
        K k = 0;
        uint32_t v = 0, d = 256u + lane;          // empty slots never match a digit
        if (valid) {
            k = FIRST ? order_key(src_t[el]) : src_k[el];
            v = FIRST ? e0 + el : src_v[el];
            d = (uint32_t)(k >> shift) & 255u;
        }
        const uint32_t vm = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
        const uint32_t peers = (e % 2 == 1 ? __match_any_sync(0xffffffffu, d) : peers8(d)) & vm;
        key[e] = k;
        val[e] = v;
        info[e] = valid ? d | ((uint32_t)__popc(peers & lt) << 8) | ((uint32_t)__popc(peers) << 16) : 0xffffffffu;
    }
#pragma unroll
    for (int e = 0; e < SLOTS; ++e) {
        const bool valid = info[e] != 0xffffffffu;
        const uint32_t d = info[e] & 255u, below = (info[e] >> 8) & 255u;
        uint32_t base = 0;
        if (valid) base = wcnt[warp][d];
        __syncwarp();
        if (valid && below == 0) wcnt[warp][d] = base + (info[e] >> 16);
        __syncwarp();
        rk[e] = valid ? base + below : 0xffffffffu;
    }
    __syncthreads();
    // per-digit prefix over warps (in place)
    uint32_t tot = 0;
    if (THREADS == 256 || tid < 256) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t v = wcnt[w][tid];
            wcnt[w][tid] = tot;
            tot += v;
        }
    }
    if (MODE == kSortArgsortScatter) {
        __syncthreads();
        // all loads of s before the thread's first store
        const T* __restrict__ s_in = (const T*)a.s_in + off;
        T* __restrict__ x_out = (T*)a.x_out + off;
        T xn[SLOTS];
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
            if (rk[e] != 0xffffffffu) {
                const uint32_t d = info[e] & 255u;
                xn[e] = s_in[gb[d] + wcnt[warp][d] + rk[e]];
            }
        }
#pragma unroll
        for (int e = 0; e < SLOTS; ++e)
            if (rk[e] != 0xffffffffu) x_out[val[e]] = xn[e];
        __syncthreads();
        return;
    }
    // the tile's digit starts (digits are threads 0..255)
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31 && (THREADS == 256 || tid < 256)) wsum[warp] = incl;
    __syncthreads();
    if (THREADS == 256 || tid < 256) {
        uint32_t woff = 0;
        for (int q = 0; q < warp; ++q) woff += wsum[q];
        const uint32_t ls = woff + incl - tot;
        ldstart[tid] = ls;
        gb[tid] -= ls;  // from here on: output index of tile position i of digit d = gb[d] + i
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < SLOTS; ++e) {
        if (rk[e] != 0xffffffffu) {
            const uint32_t d = info[e] & 255u;
            const uint32_t lp = ldstart[d] + wcnt[warp][d] + rk[e];
            sk[lp] = key[e];
            sv[lp] = val[e];
        }
    }
    __syncthreads();
    K* __restrict__ kdst = (K*)kout + off;
    uint32_t* __restrict__ vdst = vout + off;
    T* __restrict__ sdst = (T*)a.s_out + off;
    for (int i = tid; i < tl; i += THREADS) {
        const K k = sk[i];
        const uint32_t dest = gb[(uint32_t)(k >> shift) & 255u] + (uint32_t)i;
        if (MODE == 0) {
            kdst[dest] = k;
            vdst[dest] = sv[i];
        } else {
            sdst[dest] = key_value(k);
        }
    }
    __syncthreads();
}

// One pass over one tile per block: the tile's output bases come from the
// per-tile histograms and their scan.
template <typename T, bool FIRST, int MODE, int THREADS, int MINB, bool MULTI>
__global__ void __launch_bounds__(THREADS, MINB) k_sort_scatter(const __grid_constant__ LaunchSet<SortArgs> set)
{
    uint32_t blk;
    const SortArgs& a = set.pick<MULTI>(blk);
    static_assert(THREADS >= 256 && THREADS % 256 == 0, "the per-digit steps take one thread per digit");
    using K = typename key_of<T>::type;
    constexpr int WARPS = THREADS / 32;
    const int ci = (int)blk / a.tpc;
    const int t = (int)blk % a.tpc;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    __shared__ K sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint32_t wcnt[WARPS][256];
    __shared__ uint32_t ldstart[256];
    __shared__ uint32_t gb[256];
    __shared__ uint32_t wsum[8];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < WARPS * 256 / THREADS; ++q) (&wcnt[0][0])[q * THREADS + tid] = 0u;
    if (THREADS == 256 || tid < 256)
        gb[tid] = a.hist[((size_t)ci * a.tpc + t) * 256 + tid] +
                  a.cbase[((size_t)ci * a.nchunks + t / kScanChunk) * 256 + tid];
    __syncthreads();
    const uint64_t off = a.curves[c].off;
    const uint32_t e0 = (uint32_t)t * (uint32_t)a.tile_len;
    const T* src_t = (const T*)a.src + off + e0;
    const K* src_k = (const K*)a.keys_in + off + e0;
    const uint32_t* src_v = a.vals_in + off + e0;
    if (a.tile_len == kSortTile)
        sort_tile<T, FIRST, MODE, true, THREADS>(a, src_t, src_k, src_v, a.keys_out, a.vals_out, a.shift, off, e0,
                                                 a.tile_len, sk, sv, wcnt, ldstart, gb, wsum);
    else
        sort_tile<T, FIRST, MODE, false, THREADS>(a, src_t, src_k, src_v, a.keys_out, a.vals_out, a.shift, off, e0,
                                                  a.tile_len, sk, sv, wcnt, ldstart, gb, wsum);
}

// Eq. 4 (Sec. 3.2.2) from the two iterates, both in natural order: one tile
// of a curve per block reads x_{i-1} (x) and x_i (xnew, where the last sort
// pass left it), adds up (ln x_i/x_{i-1})^2 in a fixed order and moves x_i
// into x.  12 B per sample (FP32), coalesced.
template <typename T>
__global__ void __launch_bounds__(kSortThreads) k_conv_delta(const int* __restrict__ cls_curves,
                                                             const CurveDev* __restrict__ curves, int tpc,
                                                             int tile_len, const uint32_t* __restrict__ eff_iters,
                                                             const int* __restrict__ d_iter,
                                                             const T* __restrict__ xnew, T* __restrict__ x,
                                                             double* __restrict__ part)
{
    const int ci = blockIdx.x / tpc;
    const int t = blockIdx.x % tpc;
    const int c = cls_curves[ci];
    if ((uint32_t)*d_iter >= eff_iters[c]) return;
    const uint64_t base = curves[c].off + (uint64_t)t * tile_len;
    const int tid = threadIdx.x;
    T lsum = 0;
    T xn[kSlots], xo[kSlots];
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
        const int i = tid + e * kSortThreads;
        if (i < tile_len) {
            xn[e] = xnew[base + i];
            xo[e] = x[base + i];
        }
    }
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
        const int i = tid + e * kSortThreads;
        if (i < tile_len) {
            lsum += ln_ratio_sq(xn[e], xo[e]);
            x[base + i] = xn[e];
        }
    }
    // tile sum in a fixed order: warp tree, then the warps in order
    double v = (double)lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double wpart[kSortWarps];
    if ((tid & 31) == 0) wpart[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double tsum = 0.0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) tsum += wpart[w];
        part[blockIdx.x] = tsum;
    }
}

template <typename T>
void launch_conv_delta(const Plan& p, const ClassInfo& k, const void* xnew, cudaStream_t st)
{
    k_conv_delta<T><<<k.ncurves * k.tiles_per_curve, kSortThreads, 0, st>>>(
        k.d_curves, p.d_curves, k.tiles_per_curve, k.tile_len, p.d_eff_iters, p.d_iter, (const T*)xnew,
        (T*)p.d_x, p.conv.part);
}
template void launch_conv_delta<float>(const Plan&, const ClassInfo&, const void*, cudaStream_t);
template void launch_conv_delta<double>(const Plan&, const ClassInfo&, const void*, cudaStream_t);

// Eq. 4 per curve of the class: the tile sums of the last scatter in tile
// order, delta = sqrt(sum / N) / ln 10; the curve stops after this iteration
// when delta falls below its threshold.
__global__ void k_conv_finalize(const int* __restrict__ cls_curves, const CurveDev* __restrict__ curves,
                                int ncurves, int tpc, const int* __restrict__ d_iter,
                                uint32_t* __restrict__ eff_iters, ConvDev cv)
{
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncurves) return;
    const int c = cls_curves[ci];
    const int i = *d_iter;
    if ((uint32_t)i >= eff_iters[c]) return;
    double sum = 0.0;
    for (int t = 0; t < tpc; ++t) sum += cv.part[(size_t)ci * tpc + t];
    const double delta = conv_delta(sum, (double)(1ull << curves[c].log2n));
    if (conv_record(cv, c, i, delta)) eff_iters[c] = (uint32_t)i + 1u;
}

__global__ void k_conv_reset(double* __restrict__ delta, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        delta[q] = __longlong_as_double(0x7ff8000000000000ll);
}

void launch_conv_finalize(const Plan& p, const ClassInfo& k, cudaStream_t st)
{
    k_conv_finalize<<<(k.ncurves + 127) / 128, 128, 0, st>>>(k.d_curves, p.d_curves, k.ncurves, k.tiles_per_curve,
                                                             p.d_iter, p.d_eff_iters, p.conv);
}

void launch_conv_reset(const Plan& p, cudaStream_t st)
{
    const size_t n = p.ncurves * (size_t)p.conv.hist;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_conv_reset<<<blocks, 256, 0, st>>>(p.conv.delta, n);
}

// 256 threads and at most 48 registers (five blocks per SM): measured on the
// 4096 x 2^16 batch, 5.60 ms of scatter per iteration against 6.18 ms with
// 64 registers (four blocks) and 9.47 ms with 512-thread blocks.
template <typename T, bool FIRST, bool MULTI>
static void scatter_v(int mode, const LaunchSet<SortArgs>& s, uint32_t g, cudaStream_t st)
{
    constexpr int TH = 256, MB = 5;
    if (mode == 0) k_sort_scatter<T, FIRST, 0, TH, MB, MULTI><<<g, TH, 0, st>>>(s);
    else if (mode == kSortArgsortScatter) k_sort_scatter<T, FIRST, kSortArgsortScatter, TH, MB, MULTI><<<g, TH, 0, st>>>(s);
    else k_sort_scatter<T, FIRST, kSortKeysToValues, TH, MB, MULTI><<<g, TH, 0, st>>>(s);
}

template <typename T, bool FIRST>
static int launch_scatter(int mode, const std::vector<SortArgs>& args, const std::vector<uint32_t>& blocks,
                          cudaStream_t st)
{
    return for_launch_sets(args, blocks, [&](const LaunchSet<SortArgs>& s, uint32_t g, bool multi) {
        if (multi) scatter_v<T, FIRST, true>(mode, s, g, st);
        else scatter_v<T, FIRST, false>(mode, s, g, st);
    });
}

template <typename T, int TPB>
static int launch_hist_t(bool first, const std::vector<SortArgs>& args, const std::vector<uint32_t>& blocks,
                         cudaStream_t st)
{
    return for_launch_sets(args, blocks, [&](const LaunchSet<SortArgs>& s, uint32_t g, bool multi) {
        if (first && multi) k_sort_hist<T, true, TPB, true><<<g, kSortThreads, 0, st>>>(s);
        else if (first) k_sort_hist<T, true, TPB, false><<<g, kSortThreads, 0, st>>>(s);
        else if (multi) k_sort_hist<T, false, TPB, true><<<g, kSortThreads, 0, st>>>(s);
        else k_sort_hist<T, false, TPB, false><<<g, kSortThreads, 0, st>>>(s);
    });
}

// Four tiles per histogram block where a curve has them (measured on the
// 4096 x 2^16 batch: 1.25 ms of histograms and scans per iteration with one
// tile per block, 1.02 with two, 1.00 with four): the classes are grouped by
// tiles per block.
template <typename T>
static int launch_hist(bool first, const std::vector<SortArgs>& args, cudaStream_t st)
{
    std::vector<SortArgs> g[3];
    std::vector<uint32_t> b[3];
    for (const SortArgs& a : args) {
        const int tpb = std::min(4, a.tpc);
        const int q = tpb >= 4 ? 2 : (tpb >= 2 ? 1 : 0);
        g[q].push_back(a);
        b[q].push_back((uint32_t)(a.ncurves * (a.tpc / (1 << q))));
    }
    return launch_hist_t<T, 4>(first, g[2], b[2], st) + launch_hist_t<T, 2>(first, g[1], b[1], st) +
           launch_hist_t<T, 1>(first, g[0], b[0], st);
}

// Tile prefixes and digit bases: one launch for the classes whose curves
// have at most kScanChunk tiles, two (tiles, then chunks) for the others.
static int launch_scan(const std::vector<SortArgs>& args, cudaStream_t st)
{
    std::vector<SortArgs> one, two;
    std::vector<uint32_t> b_one, b_tiles, b_two;
    for (const SortArgs& a : args) {
        if (a.nchunks == 1) {
            one.push_back(a);
            b_one.push_back((uint32_t)a.ncurves);
        } else {
            two.push_back(a);
            b_tiles.push_back((uint32_t)(a.ncurves * a.nchunks));
            b_two.push_back((uint32_t)a.ncurves);
        }
    }
    int n = 0;
    n += for_launch_sets(one, b_one, [&](const LaunchSet<SortArgs>& s, uint32_t g, bool multi) {
        if (multi) k_sort_scan_curve<true><<<g, 256, 0, st>>>(s);
        else k_sort_scan_curve<false><<<g, 256, 0, st>>>(s);
    });
    n += for_launch_sets(two, b_tiles, [&](const LaunchSet<SortArgs>& s, uint32_t g, bool multi) {
        if (multi) k_sort_scan_tiles<true><<<g, 256, 0, st>>>(s);
        else k_sort_scan_tiles<false><<<g, 256, 0, st>>>(s);
    });
    n += for_launch_sets(two, b_two, [&](const LaunchSet<SortArgs>& s, uint32_t g, bool multi) {
        if (multi) k_sort_scan_chunks<true><<<g, 256, 0, st>>>(s);
        else k_sort_scan_chunks<false><<<g, 256, 0, st>>>(s);
    });
    return n;
}

template <typename T>
void launch_sort(const Plan& p, const std::vector<const ClassInfo*>& ks, const std::vector<const void*>& srcs,
                 SortMode mode, bool gated, cudaStream_t st, uint64_t* launches, void* x_out, KernelTimes* kt,
                 bool presampled)
{
    std::vector<const ClassInfo*> bk, rk;
    std::vector<const void*> bsrc, rsrc;
    for (size_t i = 0; i < ks.size(); ++i) {
        if (mode == kSortArgsortScatter && ks[i]->bucket) {
            bk.push_back(ks[i]);
            bsrc.push_back(srcs[i]);
        } else {
            rk.push_back(ks[i]);
            rsrc.push_back(srcs[i]);
        }
    }
    if (!bk.empty()) launch_bucket_argsort(p, bk, bsrc, x_out, gated, presampled, st, launches, kt);
    if (rk.empty()) return;
    using K = typename key_of<T>::type;
    const int passes = (int)sizeof(K);  // 8-bit digits
    std::vector<SortArgs> args(rk.size());
    std::vector<uint32_t> blocks(rk.size());
    for (size_t i = 0; i < rk.size(); ++i) {
        const ClassInfo& k = *rk[i];
        SortArgs& a = args[i];
        a = SortArgs{};
        a.cls_curves = k.d_curves;
        a.curves = p.d_curves;
        a.eff_iters = p.d_eff_iters;
        a.d_iter = gated ? p.d_iter : nullptr;
        a.src = rsrc[i];
        a.hist = p.d_hist + k.hist_off;
        a.cbase = p.d_cbase + k.cbase_off;
        a.x_out = x_out ? x_out : p.d_x;
        a.s_in = p.d_s;
        a.s_out = p.d_s;
        a.ncurves = k.ncurves;
        a.tpc = k.tiles_per_curve;
        a.nchunks = k.nchunks;
        a.tile_len = k.tile_len;
        blocks[i] = (uint32_t)(k.ncurves * k.tiles_per_curve);
    }
    int n = 0;
    for (int q = 0; q < passes; ++q) {
        const bool first = q == 0, last = q + 1 == passes;
        for (SortArgs& a : args) {
            a.shift = 8 * q;
            // pass q reads set (q odd ? A : B) ... with pass 0 reading `src`
            a.keys_in = (q % 2 == 1) ? p.d_keysA : p.d_keysB;
            a.vals_in = (q % 2 == 1) ? p.d_valsA : p.d_valsB;
            a.keys_out = (q % 2 == 0) ? p.d_keysA : p.d_keysB;
            a.vals_out = (q % 2 == 0) ? p.d_valsA : p.d_valsB;
        }
        if (kt) kt->begin(kGroupSortHistScan, st);
        n += launch_hist<T>(first, args, st);
        n += launch_scan(args, st);
        if (kt) kt->end(st);
        const int m = last ? (int)mode : 0;
        if (kt) kt->begin(kGroupSortScatter, st);
        if (first) n += launch_scatter<T, true>(m, args, blocks, st);
        else n += launch_scatter<T, false>(m, args, blocks, st);
        if (kt) kt->end(st);
    }
    if (launches) *launches += (uint64_t)n;
}

template <typename T>
void launch_sort(const Plan& p, const ClassInfo& k, const void* src, SortMode mode, bool gated,
                 cudaStream_t st, uint64_t* launches, void* x_out, KernelTimes* kt, bool presampled)
{
    launch_sort<T>(p, std::vector<const ClassInfo*>{&k}, std::vector<const void*>{src}, mode, gated, st, launches,
                   x_out, kt, presampled);
}

template void launch_sort<float>(const Plan&, const ClassInfo&, const void*, SortMode, bool, cudaStream_t, uint64_t*,
                                void*, KernelTimes*, bool);
template void launch_sort<double>(const Plan&, const ClassInfo&, const void*, SortMode, bool, cudaStream_t,
                                 uint64_t*, void*, KernelTimes*, bool);
template void launch_sort<float>(const Plan&, const std::vector<const ClassInfo*>&, const std::vector<const void*>&,
                                 SortMode, bool, cudaStream_t, uint64_t*, void*, KernelTimes*, bool);
template void launch_sort<double>(const Plan&, const std::vector<const ClassInfo*>&, const std::vector<const void*>&,
                                  SortMode, bool, cudaStream_t, uint64_t*, void*, KernelTimes*, bool);

}  // namespace lc

// lc_sort.cu -- segmented, stable LSD radix sort of each curve's values with the
// rank-order replacement of the E13 iteration fused into its last pass
// (Sec. 3.2.2: the values are fixed, only their order changes).
//
// Keys are the order-preserving unsigned images of the values (8-bit digits,
// 4 passes for float, 8 for double); the payload is the position k in the
// curve.  Each pass: per-tile digit histograms, a two-level scan (tiles in
// chunks, then chunks) giving every (tile, digit) its output base, and a
// stable scatter that ranks equal digits in element order (warp match +
// per-warp counts).  The last pass of an argsort writes x[k] = s[rank]
// directly instead of the sorted pairs.
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

template <typename T, bool FIRST>
__device__ __forceinline__ typename key_of<T>::type load_key(const SortArgs& a, uint64_t idx)
{
    using K = typename key_of<T>::type;
    if (FIRST) return order_key(((const T*)a.src)[idx]);
    return ((const K*)a.keys_in)[idx];
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const SortArgs a)
{
    const int ci = blockIdx.x / a.tpc;
    const int t = blockIdx.x % a.tpc;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = a.curves[c].off + (uint64_t)t * a.tile_len;
    for (int e = threadIdx.x; e < a.tile_len; e += kSortThreads) {
        const auto key = load_key<T, FIRST>(a, base + e);
        atomicAdd(&h[(uint32_t)(key >> a.shift) & 255u], 1u);
    }
    __syncthreads();
    a.hist[((size_t)ci * a.tpc + t) * 256 + threadIdx.x] = h[threadIdx.x];
}

// Exclusive prefix of every digit over the tiles of one chunk (in place) and
// the chunk totals.
__global__ void __launch_bounds__(256) k_sort_scan_tiles(const SortArgs a)
{
    const int ci = blockIdx.x / a.nchunks;
    const int ch = blockIdx.x % a.nchunks;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    const int d = threadIdx.x;
    const int t0 = ch * kScanChunk;
    const int t1 = min(a.tpc, t0 + kScanChunk);
    uint32_t run = 0;
    uint32_t* h = a.hist + (size_t)ci * a.tpc * 256 + d;
    for (int t = t0; t < t1; ++t) {
        const uint32_t v = h[(size_t)t * 256];
        h[(size_t)t * 256] = run;
        run += v;
    }
    a.cbase[((size_t)ci * a.nchunks + ch) * 256 + d] = run;
}

// Chunk prefixes, digit totals and the digit bases of one curve.
__global__ void __launch_bounds__(256) k_sort_scan_chunks(const SortArgs a)
{
    const int ci = blockIdx.x;
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

// Stable scatter of one tile.  MODE 0: sorted (key, position) pairs;
// kSortArgsortScatter: x[position] = s[rank]; kSortKeysToValues: s[rank] = value.
template <typename T, bool FIRST, int MODE>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const SortArgs a)
{
    using K = typename key_of<T>::type;
    const int ci = blockIdx.x / a.tpc;
    const int t = blockIdx.x % a.tpc;
    const int c = a.cls_curves[ci];
    if (!curve_active(a, c)) return;
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t running[256];
    __shared__ uint32_t cnt[kSortWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    dbase[tid] = a.hist[((size_t)ci * a.tpc + t) * 256 + tid] +
                 a.cbase[((size_t)ci * a.nchunks + t / kScanChunk) * 256 + tid];
    running[tid] = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) cnt[w][tid] = 0;
    __syncthreads();
    const uint64_t off = a.curves[c].off;
    const uint32_t e0 = (uint32_t)t * (uint32_t)a.tile_len;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int j0 = 0; j0 < a.tile_len; j0 += kSortThreads) {
        const bool valid = j0 + tid < a.tile_len;
        const uint32_t e = e0 + j0 + tid;
        K key = 0;
        uint32_t val = 0, d = 0, peers = 0;
        if (valid) {
            key = load_key<T, FIRST>(a, off + e);
            val = FIRST ? e : a.vals_in[off + e];
            d = (uint32_t)(key >> a.shift) & 255u;
        }
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        if (valid) peers = __match_any_sync(vmask, d);
        const bool leader = valid && (lane == __ffs(peers) - 1);
        if (leader) cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += cnt[w][d];
            const uint32_t dest = dbase[d] + running[d] + pre + __popc(peers & lt_mask);
            if (MODE == 0) {
                ((K*)a.keys_out)[off + dest] = key;
                a.vals_out[off + dest] = val;
            } else if (MODE == kSortArgsortScatter) {
                ((T*)a.x_out)[off + val] = ((const T*)a.s_in)[off + dest];
            } else {
                ((T*)a.s_out)[off + dest] = key_value(key);
            }
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) { tot += cnt[w][tid]; cnt[w][tid] = 0; }
        running[tid] += tot;
        __syncthreads();
    }
}

template <typename T, bool FIRST>
static void launch_scatter(int mode, const SortArgs& a, int blocks, cudaStream_t st)
{
    if (mode == 0) k_sort_scatter<T, FIRST, 0><<<blocks, kSortThreads, 0, st>>>(a);
    else if (mode == kSortArgsortScatter) k_sort_scatter<T, FIRST, kSortArgsortScatter><<<blocks, kSortThreads, 0, st>>>(a);
    else k_sort_scatter<T, FIRST, kSortKeysToValues><<<blocks, kSortThreads, 0, st>>>(a);
}

template <typename T>
void launch_sort(const Plan& p, const ClassInfo& k, const void* src, SortMode mode, bool gated,
                 cudaStream_t st, uint64_t* launches)
{
    using K = typename key_of<T>::type;
    const int passes = (int)sizeof(K);  // 8-bit digits
    SortArgs a{};
    a.cls_curves = k.d_curves;
    a.curves = p.d_curves;
    a.eff_iters = p.d_eff_iters;
    a.d_iter = gated ? p.d_iter : nullptr;
    a.src = src;
    a.hist = p.d_hist + k.hist_off;
    a.cbase = p.d_cbase + k.cbase_off;
    a.x_out = p.d_x;
    a.s_in = p.d_s;
    a.s_out = p.d_s;
    a.ncurves = k.ncurves;
    a.tpc = k.tiles_per_curve;
    a.nchunks = k.nchunks;
    a.tile_len = k.tile_len;
    const int blocks = k.ncurves * k.tiles_per_curve;
    for (int q = 0; q < passes; ++q) {
        const bool first = q == 0, last = q + 1 == passes;
        a.shift = 8 * q;
        // pass q reads set (q odd ? A : B) ... with pass 0 reading `src`
        a.keys_in = (q % 2 == 1) ? p.d_keysA : p.d_keysB;
        a.vals_in = (q % 2 == 1) ? p.d_valsA : p.d_valsB;
        a.keys_out = (q % 2 == 0) ? p.d_keysA : p.d_keysB;
        a.vals_out = (q % 2 == 0) ? p.d_valsA : p.d_valsB;
        if (first) k_sort_hist<T, true><<<blocks, kSortThreads, 0, st>>>(a);
        else k_sort_hist<T, false><<<blocks, kSortThreads, 0, st>>>(a);
        k_sort_scan_tiles<<<k.ncurves * k.nchunks, 256, 0, st>>>(a);
        k_sort_scan_chunks<<<k.ncurves, 256, 0, st>>>(a);
        const int m = last ? (int)mode : 0;
        if (first) launch_scatter<T, true>(m, a, blocks, st);
        else launch_scatter<T, false>(m, a, blocks, st);
        if (launches) *launches += 4;
    }
}

template void launch_sort<float>(const Plan&, const ClassInfo&, const void*, SortMode, bool, cudaStream_t, uint64_t*);
template void launch_sort<double>(const Plan&, const ClassInfo&, const void*, SortMode, bool, cudaStream_t, uint64_t*);

}  // namespace lc

// lc_internal.h -- host-side plan of the GB300 light-curve generator and the
// launchers of its kernels (one translation unit per stage).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/agnlc.h"
#include "lc_common.cuh"

namespace lc {

// Curves of one length N = 2^log2n; a launch of the multi-kernel path covers
// one class or, through a LaunchSet, several classes of one stage.
struct ClassInfo {
    uint32_t log2n = 0;
    int ncurves = 0;
    int* d_curves = nullptr;           // curve indices (device)
    std::vector<int> h_curves;
    void* d_tw = nullptr;              // e^{-2 pi i k/N}, k < N/2, element type cplx<T>
    std::vector<int> radices;          // complex FFT passes (product N/2)
    int tiles_per_curve = 0;           // sort tiles
    int tile_len = 0;
    int nchunks = 0;                   // scan chunks of tiles
    size_t hist_off = 0;               // into d_hist (u32)
    size_t cbase_off = 0;              // into d_cbase (u32)
    size_t partial_off = 0;            // into d_partial (double)
    bool resident = false;             // iterated by the fused on-chip kernel
    float* d_rx = nullptr;             // L2 exchange area of the cluster kernel (3 N floats per curve)
    bool bucket = false;               // argsort by the sample sort of lc_bucket.cu
    uint32_t* d_aux = nullptr;         // its splitters, bases and work items
    int ntab = 0;                      // curves with a tabulated ERDF (Eq. 1 smooth, Eq. 2)
    int* d_tab_curves = nullptr;       // their curve indices (device)
    std::vector<int> h_tab_curves;
};

struct Plan {
    int device = 0;
    lc_precision prec = LC_FP32;
    size_t ncurves = 0;
    size_t total = 0;        // sum N
    size_t total_h = 0;      // sum (N/2 + 1)
    uint32_t max_iters = 0;
    std::vector<lc_job> jobs;
    std::vector<CurveDev> h_curves;
    std::vector<ClassInfo> classes;

    // device memory (one arena)
    void* arena = nullptr;
    size_t arena_bytes = 0;
    CurveDev* d_curves = nullptr;
    ErdfConst* d_erdf = nullptr;
    double* d_sigma = nullptr;
    double* d_partial = nullptr;   // TK95 variance partials: realised, then (at partial_total) PSD
    size_t partial_total = 0;
    uint32_t* d_eff_iters = nullptr;
    int* d_iter = nullptr;
    void* d_x = nullptr;       // state, sum N (T)
    void* d_f = nullptr;       // FFT ping-pong, sum N (T)
    void* d_A = nullptr;       // amplitudes, sum (N/2+1) (T)
    void* d_s = nullptr;       // sorted draws, sum N (T)
    void* d_keysA = nullptr;   // sort keys (K), sum N
    void* d_keysB = nullptr;
    uint32_t* d_valsA = nullptr;
    uint32_t* d_valsB = nullptr;
    double2* d_spec = nullptr; // FP64 TK spectrum (setup only; aliases the sort buffers)
    uint32_t* d_hist = nullptr;
    uint32_t* d_cbase = nullptr;
    size_t tw_bytes = 0;
    void* d_tk_stage = nullptr;  // lazily allocated for lc_generate_host
    uint32_t* d_lags = nullptr;  // structure-function lags (kMaxLags)
    size_t ntab = 0;             // curves with a tabulated ERDF
    int* d_tab_curves = nullptr; // their indices (device)
    double* d_tab = nullptr;     // their CDF tables, kErdfTable + 1 doubles each

    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t t_setup0 = nullptr, t_setup1 = nullptr, t_it0 = nullptr, t_it1 = nullptr;
    bool timed_setup = false, timed_iter = false;
    cudaGraphExec_t iter_graph = nullptr;
    uint64_t launches_per_iter = 0;
    uint64_t last_launches = 0;
    bool setup_done = false;
    int path_mode = 0;        // 0 auto (measured table), 1 resident where possible, 2 multi-kernel
    int res_max_log2 = -1;    // auto mode: longest length on the fused kernels (-1: the built-in table)

    bool ext = false;            // state / FFT / draw / sort buffers are external planes

    // convergence test (Sec. 3.2.2, Eq. 4), off until lc_plan_set_convergence
    bool conv_on = false;
    void* conv_arena = nullptr;  // thresholds, delta record, partial sums
    ConvDev conv{};
    size_t conv_part = 0;        // doubles in conv.part
};

// CUDA events around the kernel groups of one profiled iteration.
enum KernelGroup {
    kGroupFFT = 0,           // transforms and spectral step (multi-kernel path)
    kGroupSortHistScan = 1,  // per-tile histograms and their scans
    kGroupSortScatter = 2,   // ranked scatter passes
    kGroupResident = 3,      // fused on-chip iteration kernels
    kGroupOther = 4,         // convergence test
    kGroups = 5
};
struct KernelTimes {
    struct Span {
        int group;
        cudaEvent_t a, b;
    };
    std::vector<Span> spans;
    void begin(int g, cudaStream_t st)
    {
        Span s{g, nullptr, nullptr};
        cudaEventCreate(&s.a);
        cudaEventCreate(&s.b);
        cudaEventRecord(s.a, st);
        spans.push_back(s);
    }
    void end(cudaStream_t st) { cudaEventRecord(spans.back().b, st); }
    ~KernelTimes()
    {
        for (auto& s : spans) {
            cudaEventDestroy(s.a);
            cudaEventDestroy(s.b);
        }
    }
};

// ConvDev of a plan: null pointers when the convergence test is off.
inline ConvDev conv_of(const Plan& p) { return p.conv_on ? p.conv : ConvDev{}; }

// One launch of a stage's kernel over up to kSetMax length classes: entry k
// (its own kernel arguments c[k]) owns blocks [start[k], start[k + 1]) of
// the grid, start[0] = 0.  Kernels take it as a __grid_constant__ parameter
// and have two forms: MULTI = false (one entry; c[0] is read at fixed
// offsets of the parameter space and the block index is blockIdx.x) and
// MULTI = true (the entry is found by comparing blockIdx.x with start[]).
// Both forms run the same per-block code, so a curve's results do not
// depend on the classes it is launched with.
constexpr int kSetMax = 8;
template <class A>
struct LaunchSet {
    A c[kSetMax];
    uint32_t start[kSetMax];
    int n;
#ifdef __CUDACC__
    template <bool MULTI>
    __device__ __forceinline__ const A& pick(uint32_t& bid) const
    {
        if (!MULTI) {
            bid = blockIdx.x;
            return c[0];
        }
        int k = 0;
#pragma unroll
        for (int i = 1; i < kSetMax; ++i) k += (i < n && blockIdx.x >= start[i]) ? 1 : 0;
        bid = blockIdx.x - start[k];
        return c[k];
    }
#endif
};

// Splits (args[i], blocks[i]) into launch sets of at most kSetMax entries
// (entries with no blocks are left out) and calls go(set, grid blocks,
// multi) for each; returns the number of launches.
template <class A, class F>
int for_launch_sets(const std::vector<A>& args, const std::vector<uint32_t>& blocks, F&& go)
{
    int launches = 0;
    size_t i = 0;
    while (i < args.size()) {
        LaunchSet<A> s{};
        uint32_t total = 0;
        for (; i < args.size() && s.n < kSetMax; ++i) {
            if (blocks[i] == 0) continue;
            s.c[s.n] = args[i];
            s.start[s.n] = total;
            total += blocks[i];
            ++s.n;
        }
        if (s.n == 0) continue;
        go(s, total, s.n > 1);
        ++launches;
    }
    return launches;
}

// lags of one lc_structure_function call
constexpr size_t kMaxLags = 4096;

// setup stage (lc_setup.cu)
int spec_blocks_per_curve(uint32_t log2n);
void launch_tk_spectrum(const Plan& p, const ClassInfo& k, cudaStream_t st);
template <typename T> void launch_amplitudes(const Plan& p, const ClassInfo& k, cudaStream_t st);
void launch_erdf_constants(const Plan& p, cudaStream_t st);
// CDF tables of every curve with a tabulated ERDF shape (before the draws)
void launch_erdf_tables(const Plan& p, cudaStream_t st);
template <typename T> void launch_erdf_draws(const Plan& p, const ClassInfo& k, cudaStream_t st);

// FFT stage (lc_fft.cu)
std::vector<int> fft_radices(uint32_t log2m);
// Whether the tile-path passes of a length-2^log2M transform meet the tile
// kernels' shape rules (host check at plan creation).
bool tile_schedule_ok(uint32_t log2M, bool fp64);
template <typename T> void launch_twiddles(const ClassInfo& k, cudaStream_t st);
// Complex FFT of every curve of the class (forward: e^{-}, inverse: e^{+}),
// ping-ponging between `in` and `other`; the last pass writes `final_out`
// when it is non-null.  Returns the buffer that holds the result.  When
// `gated` the kernels skip curves whose iteration budget is spent.  A
// non-null `scratch` takes the place of `in` after the first pass, so that
// `in` is only read.
template <typename T> void* launch_fft(const Plan& p, const ClassInfo& k, bool inverse, void* in,
                                       void* other, void* final_out, bool gated, cudaStream_t st,
                                       uint64_t* launches, void* scratch = nullptr);
template <typename T> void launch_spectral_iter(const Plan& p, const ClassInfo& k, const void* Z,
                                                void* Zp, cudaStream_t st);
// Forward FFT, spectral step and inverse FFT of one iteration of a tile-path
// class (log2 N >= 13) with the spectral step fused between the two
// transforms' middle passes; `in` is only read, the passes alternate between
// b and c (c may be in); returns the buffer holding x_adj.  Gated.
template <typename T> void* launch_fft_iteration(const Plan& p, const ClassInfo& k, void* in, void* b, void* c,
                                                 cudaStream_t st, uint64_t* launches);
// The same for several tile-path classes, stage by stage with one launch per
// kernel form of a stage; outs[i] receives the buffer with ks[i]'s x_adj.
template <typename T> void launch_fft_iteration(const Plan& p, const std::vector<const ClassInfo*>& ks, void* in,
                                                void* b, void* c, cudaStream_t st, uint64_t* launches,
                                                std::vector<void*>& outs);
template <typename T> void launch_spectral_tk(const Plan& p, const ClassInfo& k, void* Zp, cudaStream_t st);

// sort stage (lc_sort.cu)
constexpr int kSortTile = 2048;
constexpr int kScanChunk = 32;
enum SortMode { kSortArgsortScatter = 1, kSortKeysToValues = 2 };
// Stable LSD radix sort of each curve's values `src` (order keys of T):
// kSortArgsortScatter writes x[perm[r]] = s[r] (x = x_out, default the
// state); kSortKeysToValues writes the sorted values to s.  presampled: src
// is the iteration's x_adj, whose sample the inverse transform's last pass
// has written for the sample-sorted classes.
template <typename T> void launch_sort(const Plan& p, const ClassInfo& k, const void* src, SortMode mode,
                                       bool gated, cudaStream_t st, uint64_t* launches, void* x_out = nullptr,
                                       KernelTimes* kt = nullptr, bool presampled = false);
// The same for several classes (srcs[i]: the values of ks[i]): each kernel of
// a pass is launched once for all classes that share its form.
template <typename T> void launch_sort(const Plan& p, const std::vector<const ClassInfo*>& ks,
                                       const std::vector<const void*>& srcs, SortMode mode, bool gated,
                                       cudaStream_t st, uint64_t* launches, void* x_out, KernelTimes* kt,
                                       bool presampled);
// sample-sort argsort of the iteration (lc_bucket.cu): FP32 curves of
// 2^kBkMinLog2 .. 2^kBkMaxLog2 samples (256 buckets of N/256 elements on
// average); groups of at most bucket_cap(log2n) elements (kBkCap up to 2^18,
// N/128 above) are ranked in shared memory
constexpr int kBkCap = 2048;
constexpr uint32_t kBkMinLog2 = 13;
constexpr uint32_t kBkMaxLog2 = 20;
int bucket_samples(uint32_t log2n);  // values in the splitter sample
int bucket_cap(uint32_t log2n);      // elements of a finish group at most
bool bucket_supported(lc_precision prec, uint32_t log2n);
// LC_SORT=radix keeps the LSD radix argsort for every length
bool bucket_enabled_from_env();
int bucket_gmax(uint32_t log2n);
size_t bucket_aux_words(uint32_t log2n, int ncurves);  // u32 words of a class
cudaError_t bucket_kernel_attributes();
// x_out[perm[r]] = s[r] with perm the stable argsort of `src` (gated).
void launch_bucket_argsort(const Plan& p, const ClassInfo& k, const void* src, void* x_out, bool gated,
                           bool presampled, cudaStream_t st, uint64_t* launches, KernelTimes* kt);
// The same for several sample-sorted classes (srcs[i]: the values of
// ks[i]) with one launch per kernel for all of them.
void launch_bucket_argsort(const Plan& p, const std::vector<const ClassInfo*>& ks,
                           const std::vector<const void*>& srcs, void* x_out, bool gated, bool presampled,
                           cudaStream_t st, uint64_t* launches, KernelTimes* kt);
// where the inverse transform's last pass writes the class's samples of
// x_adj (curve ci at + ci bucket_curve_words(log2n) floats), and the shift of
// their complex index (PassArgs::smp_shift)
float* bucket_sample_area(const ClassInfo& k);
int bucket_curve_words(uint32_t log2n);
uint32_t bucket_sample_shift(uint32_t log2n);
// Eq. 4 partial sums of a multi-kernel class between the state x_{i-1} and
// the new iterate x_i in `xnew` (one double per sort tile, curve-major, in
// conv.part), moving x_i into the state; for launch_conv_finalize.
template <typename T> void launch_conv_delta(const Plan& p, const ClassInfo& k, const void* xnew, cudaStream_t st);

// fused on-chip iteration (lc_resident.cu)
bool resident_supported(const Plan& p, uint32_t log2n);
// path mode from the environment: LC_PATH=resident -> 1, multi -> 2, else 0 (auto)
int path_mode_from_env();
// LC_RESIDENT_MAX_LOG2 (9..16: the longest length the auto mode runs on the
// fused kernels; 9 = none), else -1
int resident_max_log2_from_env();
// floats of cluster exchange area per curve of length 2^log2n (0: none needed)
size_t resident_exchange_floats(uint32_t log2n);
// Runs n_it iterations (from the plan's current iteration index) of every
// curve of a resident class in one launch.
void launch_resident(const Plan& p, const ClassInfo& k, uint32_t n_it, cudaStream_t st, uint64_t* launches);

// Eq. 4 per curve of a multi-kernel class from the tile partial sums of the
// last scatter; records delta and stops the curves that fell below threshold.
void launch_conv_finalize(const Plan& p, const ClassInfo& k, cudaStream_t st);
// Marks the whole delta record "not run" (NaN).
void launch_conv_reset(const Plan& p, cudaStream_t st);

void launch_iter_increment(const Plan& p, cudaStream_t st);
void launch_iter_add(const Plan& p, uint32_t n, cudaStream_t st);
void launch_eff_iters(const Plan& p, uint32_t override_iters, cudaStream_t st);

// Kernel attributes that are set once per device before the first launch
// (dynamic shared-memory limits of the tile FFT and fused kernels); the
// device must be current.  LC_ERR_CUDA with the error text on failure.
cudaError_t fft_kernel_attributes();
cudaError_t resident_kernel_attributes();
lc_status prepare_kernels(int device);

void set_error(const std::string& msg);
const char* last_error_text();
lc_status validate_job(const lc_job& j);
// Curve descriptor of a job (offsets, class and table offset left to the caller).
CurveDev curve_from_job(const lc_job& j);

// plan life cycle shared by the batch ABI and the server
lc_status plan_create(const lc_job* jobs, size_t njobs, lc_precision prec, int device, Plan** out);
// Large per-sample buffers owned by someone else (the server): curve c of a
// plan built on them uses samples [off_c, off_c + N_c) of x, f, s, the key and
// position planes, and entries [h_c, h_c + N_c/2 + 1) of A and spec, h_c =
// ext_half_offset(off_c).  off_c must be a multiple of N_c (>= 16), so that
// the half ranges of curves whose sample ranges are disjoint are disjoint.
struct ExtPlanes {
    void* x;
    void* f;
    void* A;
    void* s;
    void* keysA;
    void* keysB;
    uint32_t* valsA;
    uint32_t* valsB;
    double2* spec;
};
size_t ext_half_offset(uint64_t off);
// bytes of the external planes per sample of capacity
size_t ext_plane_bytes_per_sample(lc_precision prec);
lc_status plan_create_ext(const lc_job* jobs, size_t njobs, lc_precision prec, int device, const ExtPlanes* ext,
                          const uint64_t* ext_off, Plan** out);
// device bytes plan_create (ext = false) or plan_create_ext (ext = true)
// allocates for these jobs; no device call
lc_status plan_arena_bytes(const lc_job* jobs, size_t njobs, lc_precision prec, bool ext, size_t* bytes);
lc_status plan_setup(Plan& p, void* out_tk, cudaStream_t st, uint64_t* launches);
// n_it more iterations from the current iteration index (each curve stops at
// its own job count)
lc_status plan_continue(Plan& p, uint32_t n_it, cudaStream_t st, uint64_t* launches);
void plan_free(Plan* p);

// host helpers of the entry points
#define LC_CK(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ::lc::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return LC_ERR_CUDA;                                                              \
        }                                                                                    \
    } while (0)

// makes `dev` current for the scope of the guard
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// orders the plan's stream after the caller's stream on entry and the
// caller's stream after the plan's on exit
struct StreamJoin {
    Plan& p;
    cudaStream_t user;
    StreamJoin(Plan& pl, void* s) : p(pl), user((cudaStream_t)s)
    {
        cudaEventRecord(p.ev_in, user);
        cudaStreamWaitEvent(p.stream, p.ev_in, 0);
    }
    ~StreamJoin()
    {
        cudaEventRecord(p.ev_out, p.stream);
        cudaStreamWaitEvent(user, p.ev_out, 0);
    }
};

}  // namespace lc

// the opaque handle of the C ABI
struct lc_plan_s : public lc::Plan {};

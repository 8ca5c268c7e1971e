// lc_noalloc.cu -- single-curve generator entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: embedders whose device memory is owned
// by another allocator (a framework's caching allocator or a memory pool that
// must account for every byte), and real-time or serving loops that forbid
// allocation after start-up because a cudaMalloc can synchronise the device
// and stall unrelated work.  lc_generate_noalloc runs the whole generator for
// one FP32 curve of up to 2^16 samples with every intermediate buffer carved
// from one file-scope device array; the caller passes only the job and the
// output.
#include <mutex>

#include "lc_internal.h"

namespace lc {

// Scratch of the allocation-free entry point: 4 MiB, enough for one FP32 curve
// of 2^16 samples (state, FFT ping-pong, amplitudes, sorted draws, sort keys
// and positions, histograms, twiddles, descriptors).  Every device that loads
// the library holds it until the process exits.
constexpr size_t kNoallocBytes = (size_t)4 << 20;
constexpr uint32_t kNoallocMaxLog2 = 16;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[128];

// Device address of the scratch array on the current device (looked up once
// per device; the symbol name is only a host-side handle).
static lc_status noalloc_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= 128) { set_error("device ordinal out of range"); return LC_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return LC_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LC_OK;
}

static size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Writes the curve descriptor and the class's curve index from kernel
// arguments (copied at launch), so no host memory is read after the call.
__global__ void k_noalloc_descriptors(CurveDev cv, CurveDev* __restrict__ d_cv, int* __restrict__ d_cls)
{
    *d_cv = cv;
    *d_cls = 0;
}

}  // namespace lc

using namespace lc;

extern "C" lc_status lc_generate_noalloc(const lc_job* job, void* out_x, void* stream)
{
    if (!job || !out_x) { set_error("null job or out_x"); return LC_ERR_INVALID; }
    lc_status st = validate_job(*job);
    if (st != LC_OK) return st;
    if (job->log2n > kNoallocMaxLog2) {
        set_error("lc_generate_noalloc: log2n above 16 exceeds the 4 MiB static scratch");
        return LC_ERR_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); set_error("no current CUDA device"); return LC_ERR_CUDA; }
    st = prepare_kernels(dev);
    if (st != LC_OK) return st;
    void* base = nullptr;
    st = noalloc_scratch(dev, &base);
    if (st != LC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // one-curve plan whose buffers live in the static scratch
    Plan p;
    p.device = dev;
    p.prec = LC_FP32;
    p.ncurves = 1;
    p.path_mode = path_mode_from_env();
    p.res_max_log2 = resident_max_log2_from_env();
    const size_t n = (size_t)1 << job->log2n, nh = n / 2 + 1, ts = 4;
    CurveDev cv = curve_from_job(*job);
    cv.off = 0; cv.offh = 0; cv.cls = 0; cv.tab = 0;
    const bool tabulated = cv.kind != LC_ERDF_SHARP;
    p.h_curves.assign(1, cv);
    p.total = n; p.total_h = nh; p.max_iters = job->iters;
    p.classes.emplace_back();
    ClassInfo& k = p.classes.back();
    k.log2n = job->log2n;
    k.ncurves = 1;
    k.h_curves.assign(1, 0);
    k.radices = fft_radices(k.log2n - 1);
    k.tile_len = (int)(n < (size_t)kSortTile ? n : (size_t)kSortTile);
    k.tiles_per_curve = (int)(n / k.tile_len);
    k.nchunks = (k.tiles_per_curve + kScanChunk - 1) / kScanChunk;
    k.resident = resident_supported(p, k.log2n);

    char* b = (char*)base;
    size_t at = 0;
    auto take = [&](size_t bytes) { char* q = b + at; at = up256(at + bytes); return (void*)q; };
    p.d_curves = (CurveDev*)take(sizeof(CurveDev));
    p.d_erdf = (ErdfConst*)take(sizeof(ErdfConst));
    p.d_sigma = (double*)take(sizeof(double) * 2);
    p.d_eff_iters = (uint32_t*)take(sizeof(uint32_t));
    p.d_iter = (int*)take(4 * sizeof(int));
    p.d_partial = (double*)take(sizeof(double) * 2 * (size_t)spec_blocks_per_curve(k.log2n));
    p.partial_total = (size_t)spec_blocks_per_curve(k.log2n);
    p.d_x = take(n * ts);
    p.d_f = take(n * ts);
    p.d_A = take(nh * ts);
    p.d_s = take(n * ts);
    const size_t sortbytes = std::max(2 * n * ts + 2 * n * 4, 16 * nh);
    char* sortb = (char*)take(sortbytes);
    p.d_keysA = sortb;
    p.d_keysB = sortb + n * ts;
    p.d_valsA = (uint32_t*)(sortb + 2 * n * ts);
    p.d_valsB = (uint32_t*)(sortb + 2 * n * ts + n * 4);
    p.d_spec = (double2*)sortb;
    p.d_hist = (uint32_t*)take(sizeof(uint32_t) * (size_t)k.tiles_per_curve * 256);
    p.d_cbase = (uint32_t*)take(sizeof(uint32_t) * (size_t)k.nchunks * 256);
    k.d_tw = take((n / 2) * 2 * ts);
    k.d_curves = (int*)take(sizeof(int));
    if (resident_exchange_floats(k.log2n)) k.d_rx = (float*)take(resident_exchange_floats(k.log2n) * 4);
    k.bucket = bucket_enabled_from_env() && bucket_supported(LC_FP32, k.log2n);
    if (k.bucket) k.d_aux = (uint32_t*)take(bucket_aux_words(k.log2n, 1) * 4);
    if (tabulated) {
        // the CDF table of a smooth (Eq. 1) or log-normal (Eq. 2) ERDF
        p.ntab = 1;
        k.ntab = 1;
        p.d_tab = (double*)take(sizeof(double) * (kErdfTable + 1));
        p.d_tab_curves = k.d_curves;  // the one curve, index 0
        k.d_tab_curves = k.d_curves;
    }
    if (at > kNoallocBytes) { set_error("lc_generate_noalloc: layout exceeds the static scratch"); return LC_ERR_INVALID; }

    k_noalloc_descriptors<<<1, 1, 0, s>>>(cv, p.d_curves, k.d_curves);
    launch_twiddles<float>(k, s);
    // setup: TK95 spectrum and amplitudes, ERDF draws, sorted draws (Sec. 2.1)
    launch_eff_iters(p, 0, s);
    launch_tk_spectrum(p, k, s);
    launch_amplitudes<float>(p, k, s);
    launch_erdf_constants(p, s);
    launch_erdf_tables(p, s);
    launch_erdf_draws<float>(p, k, s);
    launch_sort<float>(p, k, p.d_x, kSortKeysToValues, false, s, nullptr);
    // iterations (Sec. 3.2.2), launched directly (no graph)
    if (job->iters > 0) {
        if (k.resident) {
            launch_resident(p, k, job->iters, s, nullptr);
        } else {
            for (uint32_t it = 0; it < job->iters; ++it) {
                void* R3;
                if (k.log2n - 1 >= 12) {
                    R3 = launch_fft_iteration<float>(p, k, p.d_x, p.d_f, p.d_x, s, nullptr);
                } else {
                    void* R1 = launch_fft<float>(p, k, false, p.d_x, p.d_f, nullptr, true, s, nullptr);
                    void* Zp = (R1 == p.d_x) ? p.d_f : p.d_x;
                    launch_spectral_iter<float>(p, k, R1, Zp, s);
                    R3 = launch_fft<float>(p, k, true, Zp, R1, nullptr, true, s, nullptr);
                }
                launch_sort<float>(p, k, R3, kSortArgsortScatter, true, s, nullptr, nullptr, nullptr,
                                   k.log2n - 1 >= 12);
                launch_iter_increment(p, s);
            }
        }
    }
    if (cudaMemcpyAsync(out_x, p.d_x, n * ts, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        set_error("output copy failed");
        return LC_ERR_CUDA;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("lc_generate_noalloc: ") + cudaGetErrorString(e)); return LC_ERR_CUDA; }
    return LC_OK;
}

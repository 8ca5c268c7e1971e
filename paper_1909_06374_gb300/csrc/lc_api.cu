// lc_api.cu -- plans and the batch entry points of the C ABI (agnlc.h).
//
// A plan lays a batch of curves out in flat ragged buffers (curve c at
// sum_{c'<c} N_{c'}), groups curves of equal length into classes, and owns one
// device arena holding the state, the target amplitudes, the sorted draws, the
// FFT and sort scratch and the twiddle tables.  lc_setup runs the TK95 and
// ERDF stages (Sec. 2.1, steps one and two); lc_iterate replays one captured
// CUDA graph per amplitude-adjustment iteration (Sec. 3.2.2).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>

#include "lc_internal.h"

namespace lc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_text() { return g_last_error.c_str(); }


__global__ void k_iter_increment(int* d_iter) { ++*d_iter; }

__global__ void k_eff_iters(const CurveDev* __restrict__ curves, int n, uint32_t override_iters,
                            uint32_t* __restrict__ eff, int* __restrict__ d_iter)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) eff[c] = override_iters ? override_iters : curves[c].iters;
    if (c == 0) *d_iter = 0;
}

__global__ void k_iter_add(int* d_iter, uint32_t n) { *d_iter += (int)n; }

void launch_iter_increment(const Plan& p, cudaStream_t st) { k_iter_increment<<<1, 1, 0, st>>>(p.d_iter); }
void launch_iter_add(const Plan& p, uint32_t n, cudaStream_t st) { k_iter_add<<<1, 1, 0, st>>>(p.d_iter, n); }

void launch_eff_iters(const Plan& p, uint32_t override_iters, cudaStream_t st)
{
    k_eff_iters<<<(int)((p.ncurves + 255) / 256), 256, 0, st>>>(p.d_curves, (int)p.ncurves, override_iters,
                                                                p.d_eff_iters, p.d_iter);
}

lc_status prepare_kernels(int device)
{
    static std::mutex mu;
    static bool done[128];
    if (device < 0 || device >= 128) { set_error("device ordinal out of range"); return LC_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(mu);
    if (done[device]) return LC_OK;
    cudaError_t e = fft_kernel_attributes();
    if (e == cudaSuccess) e = resident_kernel_attributes();
    if (e == cudaSuccess) e = bucket_kernel_attributes();
    if (e != cudaSuccess) {
        set_error(std::string("kernel attributes: ") + cudaGetErrorString(e));
        return LC_ERR_CUDA;
    }
    done[device] = true;
    return LC_OK;
}

static bool finite(double v) { return std::isfinite(v); }

lc_status validate_job(const lc_job& j)
{
    if (j.log2n < 4 || j.log2n > 27) { set_error("log2n must be in [4, 27]"); return LC_ERR_INVALID; }
    if (!(j.dt > 0) || !finite(j.dt)) { set_error("dt must be > 0"); return LC_ERR_INVALID; }
    if (!(j.psd.f_br > 0) || !finite(j.psd.f_br)) { set_error("f_br must be > 0"); return LC_ERR_INVALID; }
    if (!finite(j.psd.alpha_low) || !finite(j.psd.alpha_high)) { set_error("PSD slopes must be finite"); return LC_ERR_INVALID; }
    if (j.psd.coeffs < LC_TK_GAUSSIAN || j.psd.coeffs > LC_TK_FIXED_AMPLITUDE) { set_error("unknown TK coefficient mode"); return LC_ERR_INVALID; }
    if (j.psd.targets < LC_TARGETS_REALISED || j.psd.targets > LC_TARGETS_PSD) { set_error("unknown target amplitude mode"); return LC_ERR_INVALID; }
    const lc_erdf& e = j.erdf;
    if (e.kind < LC_ERDF_SHARP || e.kind > LC_ERDF_LOGNORMAL) { set_error("unknown ERDF kind"); return LC_ERR_INVALID; }
    if (!finite(e.log_lmin) || !finite(e.log_lmax) || !finite(e.log_lbreak) || !finite(e.slope_low) ||
        !finite(e.slope_high)) { set_error("ERDF parameters must be finite"); return LC_ERR_INVALID; }
    if (!(e.log_lmin < e.log_lmax)) { set_error("ERDF needs log_lmin < log_lmax"); return LC_ERR_INVALID; }
    if (e.log_lmin < -300 || e.log_lmax > 300) { set_error("ERDF range out of [1e-300, 1e300]"); return LC_ERR_INVALID; }
    if (e.kind == LC_ERDF_LOGNORMAL) {
        // the table resolves the bell (>= 4 intervals per sigma) and holds mass
        if (!finite(e.sigma) || !(e.sigma >= (e.log_lmax - e.log_lmin) / 1024.0)) {
            set_error("log-normal ERDF needs sigma >= (log_lmax - log_lmin)/1024"); return LC_ERR_INVALID;
        }
        if (e.log_lbreak < e.log_lmin - 30.0 * e.sigma || e.log_lbreak > e.log_lmax + 30.0 * e.sigma) {
            set_error("log-normal ERDF centre more than 30 sigma outside the range"); return LC_ERR_INVALID;
        }
        return LC_OK;
    }
    if (!(e.log_lmin < e.log_lbreak && e.log_lbreak < e.log_lmax)) {
        set_error("ERDF needs log_lmin < log_lbreak < log_lmax"); return LC_ERR_INVALID;
    }
    if (std::fabs(e.slope_low) > 50 || std::fabs(e.slope_high) > 50) { set_error("ERDF slope magnitude > 50"); return LC_ERR_INVALID; }
    return LC_OK;
}

CurveDev curve_from_job(const lc_job& j)
{
    CurveDev cv{};
    cv.log2n = j.log2n; cv.iters = j.iters;
    cv.dt = j.dt; cv.f_br = j.psd.f_br; cv.a_lo = j.psd.alpha_low; cv.a_hi = j.psd.alpha_high;
    cv.umin = j.erdf.log_lmin; cv.umax = j.erdf.log_lmax; cv.ub = j.erdf.log_lbreak;
    cv.sl_lo = j.erdf.slope_low; cv.sl_hi = j.erdf.slope_high; cv.lin = j.erdf.linear_space ? 1 : 0;
    cv.kind = j.erdf.kind;
    cv.coeffs = j.psd.coeffs;
    cv.targets = j.psd.targets;
    cv.sigma = j.erdf.kind == LC_ERDF_LOGNORMAL ? j.erdf.sigma : 0.0;
    cv.seed = j.seed; cv.curve_id = j.curve_id;
    return cv;
}

int path_mode_from_env()
{
    const char* e = std::getenv("LC_PATH");
    if (!e) return 0;
    if (std::strcmp(e, "resident") == 0) return 1;
    if (std::strcmp(e, "multi") == 0) return 2;
    return 0;
}

int resident_max_log2_from_env()
{
    const char* e = std::getenv("LC_RESIDENT_MAX_LOG2");
    if (!e) return -1;
    char* end = nullptr;
    const long v = std::strtol(e, &end, 10);
    if (end == e || *end != 0 || v < 9 || v > 16) return -1;
    return (int)v;
}

// Everything of a plan that needs no device: validation, curve descriptors
// and offsets (in job order, or at the given external offsets), classes and
// their per-class sizes.
static lc_status plan_describe(const lc_job* jobs, size_t njobs, lc_precision prec, const uint64_t* ext_off,
                               Plan& P)
{
    if (!jobs || njobs == 0) { set_error("null jobs or njobs == 0"); return LC_ERR_INVALID; }
    if (prec != LC_FP32 && prec != LC_FP64) { set_error("bad precision"); return LC_ERR_INVALID; }
    for (size_t i = 0; i < njobs; ++i) {
        lc_status s = validate_job(jobs[i]);
        if (s != LC_OK) { set_error("job " + std::to_string(i) + ": " + g_last_error); return s; }
    }
    Plan* p = &P;
    p->prec = prec;
    p->ncurves = njobs;
    // Path selection (a tuning knob; results depend only on length,
    // precision and the path, never on the batch): LC_PATH=multi forces the
    // multi-kernel iteration everywhere, LC_PATH=resident uses the fused
    // kernels wherever they apply, the default follows the per-length table
    // measured by the autotuning sweep (autotune.py), whose crossover
    // LC_RESIDENT_MAX_LOG2 overrides.
    p->path_mode = path_mode_from_env();
    p->res_max_log2 = resident_max_log2_from_env();
    p->jobs.assign(jobs, jobs + njobs);
    // curves in job order; classes by length
    p->h_curves.resize(njobs);
    size_t off = 0, offh = 0;
    std::vector<int> cls_of_len(28, -1);
    for (size_t c = 0; c < njobs; ++c) {
        const lc_job& j = jobs[c];
        CurveDev& cv = p->h_curves[c];
        cv = curve_from_job(j);
        if (ext_off) {
            cv.off = ext_off[c];
            cv.offh = ext_half_offset(cv.off);
        } else {
            cv.off = off;
            cv.offh = offh;
        }
        if (cls_of_len[j.log2n] < 0) {
            cls_of_len[j.log2n] = (int)p->classes.size();
            p->classes.emplace_back();
            p->classes.back().log2n = j.log2n;
        }
        cv.cls = cls_of_len[j.log2n];
        p->classes[cv.cls].h_curves.push_back((int)c);
        if (cv.kind != LC_ERDF_SHARP) {
            cv.tab = (uint64_t)p->ntab * (kErdfTable + 1);
            ++p->ntab;
            p->classes[cv.cls].h_tab_curves.push_back((int)c);
        }
        off += 1ull << j.log2n;
        offh += (1ull << (j.log2n - 1)) + 1;
        p->max_iters = std::max(p->max_iters, j.iters);
    }
    p->total = off;
    p->total_h = offh;
    for (auto& k : p->classes) {
        if (k.log2n - 1 >= 12 && !tile_schedule_ok(k.log2n - 1, prec == LC_FP64)) {
            set_error("internal: no tile schedule for log2n = " + std::to_string(k.log2n));
            return LC_ERR_INVALID;
        }
    }
    const bool bucket_on = bucket_enabled_from_env();
    for (auto& k : p->classes) {
        k.ncurves = (int)k.h_curves.size();
        k.bucket = bucket_on && bucket_supported(prec, k.log2n);
        k.radices = fft_radices(k.log2n - 1);
        const size_t n = 1ull << k.log2n;
        k.tile_len = (int)std::min<size_t>(n, kSortTile);
        k.tiles_per_curve = (int)(n / k.tile_len);
        k.nchunks = (k.tiles_per_curve + kScanChunk - 1) / kScanChunk;
        k.resident = resident_supported(*p, k.log2n);
    }
    return LC_OK;
}

// Byte offsets of a plan's device arena.  With external planes the state,
// FFT, amplitude, draw and sort buffers live there instead (at the curves'
// own offsets) and the arena holds only the per-plan tables.
struct PlanLayout {
    size_t bytes = 0;
    size_t curves, erdf, sigma, eff, iter, partial, x, f, A, s, sort, hist, cbase, tw, cls, lags, tabc, tab, rx, aux;
    size_t nhist = 0, ncbase = 0, npartial = 0;
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static PlanLayout plan_layout(Plan& P, bool ext)
{
    Plan* p = &P;
    const size_t ts = p->prec == LC_FP32 ? 4 : 8;
    const size_t njobs = p->ncurves;
    PlanLayout L;
    size_t hist = 0, cbase = 0, partial = 0, twb = 0, rxb = 0, auxb = 0;
    for (auto& k : p->classes) {
        const size_t n = 1ull << k.log2n;
        if (k.bucket) auxb += align_up(bucket_aux_words(k.log2n, k.ncurves) * 4, 256);
        k.hist_off = hist;  hist += (size_t)k.ncurves * k.tiles_per_curve * 256;
        k.cbase_off = cbase; cbase += (size_t)k.ncurves * k.nchunks * 256;
        k.partial_off = partial; partial += (size_t)k.ncurves * spec_blocks_per_curve(k.log2n);
        twb += align_up((n / 2) * 2 * ts, 256);
        rxb += align_up((size_t)k.ncurves * resident_exchange_floats(k.log2n) * 4, 256);
    }
    L.nhist = hist; L.ncbase = cbase; L.npartial = partial;
    size_t sz = 0;
    auto take = [&](size_t bytes) { size_t o = sz; sz = align_up(sz + bytes, 256); return o; };
    L.curves = take(sizeof(CurveDev) * njobs);
    L.erdf = take(sizeof(ErdfConst) * njobs);
    L.sigma = take(sizeof(double) * 2 * njobs);  // realised, then PSD
    L.eff = take(sizeof(uint32_t) * njobs);
    L.iter = take(sizeof(int) * 4);
    L.partial = take(sizeof(double) * 2 * partial);
    if (!ext) {
        L.x = take(p->total * ts);
        L.f = take(p->total * ts);
        L.A = take(p->total_h * ts);
        L.s = take(p->total * ts);
        L.sort = take(std::max(2 * p->total * ts + 2 * p->total * 4, 16 * p->total_h));
    } else {
        L.x = L.f = L.A = L.s = L.sort = 0;
    }
    L.hist = take(sizeof(uint32_t) * hist);
    L.cbase = take(sizeof(uint32_t) * cbase);
    L.tw = take(twb);
    L.cls = take(sizeof(int) * njobs);
    L.lags = take(sizeof(uint32_t) * kMaxLags);
    L.tabc = take(sizeof(int) * 2 * p->ntab);  // all, then per class
    L.tab = take(sizeof(double) * (kErdfTable + 1) * p->ntab);
    L.rx = p->prec == LC_FP32 ? take(rxb) : 0;
    L.aux = take(auxb);
    L.bytes = sz;
    return L;
}

size_t ext_half_offset(uint64_t off) { return (size_t)(off / 2 + off / 16); }

size_t ext_plane_bytes_per_sample(lc_precision prec)
{
    const size_t ts = prec == LC_FP32 ? 4 : 8;
    // x, f, s, two key and two position planes; amplitudes and the FP64 TK
    // spectrum at the half offsets (9/16 of an entry per sample)
    return 5 * ts + 2 * 4 + (ts * 9 + 15) / 16 + 9;
}

lc_status plan_arena_bytes(const lc_job* jobs, size_t njobs, lc_precision prec, bool ext, size_t* bytes)
{
    Plan p;
    std::vector<uint64_t> offs;
    if (ext) {
        uint64_t o = 0;
        for (size_t i = 0; i < njobs; ++i) { offs.push_back(o); o += 1ull << (jobs ? jobs[i].log2n : 0); }
    }
    lc_status st = plan_describe(jobs, njobs, prec, ext ? offs.data() : nullptr, p);
    if (st != LC_OK) return st;
    *bytes = plan_layout(p, ext).bytes;
    return LC_OK;
}

template <typename T>
static lc_status build_tables(Plan& p)
{
    for (auto& k : p.classes) launch_twiddles<T>(k, p.stream);
    LC_CK(cudaGetLastError());
    return LC_OK;
}

lc_status plan_create_ext(const lc_job* jobs, size_t njobs, lc_precision prec, int device, const ExtPlanes* ext,
                          const uint64_t* ext_off, Plan** out)
{
    if (!out) { set_error("out is null"); return LC_ERR_INVALID; }
    if (ext && !ext_off) { set_error("external planes need the curves' offsets"); return LC_ERR_INVALID; }
    Plan* p = new (std::nothrow) Plan();
    if (!p) return LC_ERR_NOMEM;
    {
        const lc_status ds = plan_describe(jobs, njobs, prec, ext ? ext_off : nullptr, *p);
        if (ds != LC_OK) { delete p; return ds; }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete p;
        set_error("no such CUDA device"); return LC_ERR_INVALID;
    }
    DeviceGuard g(device);
    {
        const lc_status ps = prepare_kernels(device);
        if (ps != LC_OK) { delete p; return ps; }
    }
    p->device = device;
    p->ext = ext != nullptr;
    const size_t ts = prec == LC_FP32 ? 4 : 8;
    const PlanLayout L = plan_layout(*p, p->ext);
    p->arena_bytes = L.bytes;
    p->partial_total = L.npartial;
    cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_error(std::string("stream: ") + cudaGetErrorString(e)); delete p; return LC_ERR_CUDA; }
    // with external planes the arena is stream-ordered (no device-wide
    // synchronisation when a server starts or ends a cohort)
    e = p->ext ? cudaMallocAsync(&p->arena, L.bytes, p->stream) : cudaMalloc(&p->arena, L.bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of " + std::to_string(L.bytes) + " bytes failed");
        cudaStreamDestroy(p->stream);
        delete p;
        return LC_ERR_NOMEM;
    }
    char* base = (char*)p->arena;
    p->d_curves = (CurveDev*)(base + L.curves);
    p->d_erdf = (ErdfConst*)(base + L.erdf);
    p->d_sigma = (double*)(base + L.sigma);
    p->d_eff_iters = (uint32_t*)(base + L.eff);
    p->d_iter = (int*)(base + L.iter);
    p->d_partial = (double*)(base + L.partial);
    p->d_lags = (uint32_t*)(base + L.lags);
    if (p->ext) {
        p->d_x = ext->x;
        p->d_f = ext->f;
        p->d_A = ext->A;
        p->d_s = ext->s;
        p->d_keysA = ext->keysA;
        p->d_keysB = ext->keysB;
        p->d_valsA = ext->valsA;
        p->d_valsB = ext->valsB;
        p->d_spec = ext->spec;
    } else {
        p->d_x = base + L.x;
        p->d_f = base + L.f;
        p->d_A = base + L.A;
        p->d_s = base + L.s;
        p->d_keysA = base + L.sort;
        p->d_keysB = base + L.sort + p->total * ts;
        p->d_valsA = (uint32_t*)(base + L.sort + 2 * p->total * ts);
        p->d_valsB = (uint32_t*)(base + L.sort + 2 * p->total * ts + p->total * 4);
        p->d_spec = (double2*)(base + L.sort);
    }
    p->d_hist = (uint32_t*)(base + L.hist);
    p->d_cbase = (uint32_t*)(base + L.cbase);
    size_t tw_at = L.tw, cls_at = L.cls, rx_at = L.rx, aux_at = L.aux;
    size_t twb = 0;
    for (auto& k : p->classes) {
        if (k.bucket) {
            k.d_aux = (uint32_t*)(base + aux_at);
            aux_at += align_up(bucket_aux_words(k.log2n, k.ncurves) * 4, 256);
        }
        k.d_tw = base + tw_at;
        tw_at += align_up((((size_t)1 << k.log2n) / 2) * 2 * ts, 256);
        twb += align_up((((size_t)1 << k.log2n) / 2) * 2 * ts, 256);
        k.d_curves = (int*)(base + cls_at);
        cls_at += sizeof(int) * k.h_curves.size();
        const size_t rx = prec == LC_FP32 ? (size_t)k.ncurves * resident_exchange_floats(k.log2n) * 4 : 0;
        if (rx) {
            k.d_rx = (float*)(base + rx_at);
            rx_at += align_up(rx, 256);
        }
    }
    p->tw_bytes = twb;
    std::vector<int> tab_all, tab_cls;
    if (p->ntab) {
        p->d_tab = (double*)(base + L.tab);
        p->d_tab_curves = (int*)(base + L.tabc);
        for (size_t c = 0; c < njobs; ++c)
            if (p->h_curves[c].kind != LC_ERDF_SHARP) tab_all.push_back((int)c);
        for (auto& k : p->classes) {
            k.ntab = (int)k.h_tab_curves.size();
            k.d_tab_curves = p->d_tab_curves + p->ntab + tab_cls.size();
            tab_cls.insert(tab_cls.end(), k.h_tab_curves.begin(), k.h_tab_curves.end());
        }
        tab_all.insert(tab_all.end(), tab_cls.begin(), tab_cls.end());
    }

    auto fail = [&](const char* what, cudaError_t e2) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e2));
        if (p->ext) cudaFreeAsync(p->arena, p->stream);
        else cudaFree(p->arena);
        cudaStreamSynchronize(p->stream);
        cudaStreamDestroy(p->stream);
        delete p;
        return LC_ERR_CUDA;
    };
    cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming);
    cudaEventCreate(&p->t_setup0);
    cudaEventCreate(&p->t_setup1);
    cudaEventCreate(&p->t_it0);
    cudaEventCreate(&p->t_it1);
    if ((e = cudaMemcpyAsync(p->d_curves, p->h_curves.data(), sizeof(CurveDev) * njobs, cudaMemcpyHostToDevice,
                             p->stream)) != cudaSuccess) return fail("upload curves", e);
    for (auto& k : p->classes) {
        if ((e = cudaMemcpyAsync(k.d_curves, k.h_curves.data(), sizeof(int) * k.h_curves.size(),
                                 cudaMemcpyHostToDevice, p->stream)) != cudaSuccess) return fail("upload classes", e);
    }
    if (p->ntab && (e = cudaMemcpyAsync(p->d_tab_curves, tab_all.data(), sizeof(int) * tab_all.size(),
                                        cudaMemcpyHostToDevice, p->stream)) != cudaSuccess)
        return fail("upload table curves", e);
    lc_status st = prec == LC_FP32 ? build_tables<float>(*p) : build_tables<double>(*p);
    if (st != LC_OK) return fail("twiddle tables", cudaGetLastError());
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return fail("plan sync", e);
    *out = p;
    return LC_OK;
}

lc_status plan_create(const lc_job* jobs, size_t njobs, lc_precision prec, int device, Plan** out)
{
    return plan_create_ext(jobs, njobs, prec, device, nullptr, nullptr, out);
}

// ------------------------------------------------------------ stages
template <typename T>
static lc_status run_setup(Plan& p, void* out_tk, cudaStream_t st, uint64_t* launches)
{
    cudaEventRecord(p.t_setup0, st);
    p.timed_setup = true;
    p.timed_iter = false;
    launch_eff_iters(p, 0, st);
    ++*launches;
    for (auto& k : p.classes) { launch_tk_spectrum(p, k, st); *launches += 2; }
    for (auto& k : p.classes) { launch_amplitudes<T>(p, k, st); ++*launches; }
    if (out_tk) {
        for (auto& k : p.classes) {
            launch_spectral_tk<T>(p, k, p.d_f, st);
            ++*launches;
            launch_fft<T>(p, k, true, p.d_f, p.d_x, out_tk, false, st, launches);
        }
    }
    launch_erdf_constants(p, st);
    ++*launches;
    if (p.ntab) {
        launch_erdf_tables(p, st);
        ++*launches;
    }
    for (auto& k : p.classes) { launch_erdf_draws<T>(p, k, st); *launches += (k.ntab < k.ncurves) + (k.ntab > 0); }
    {
        // the draws of every class sorted with one launch per kernel form
        std::vector<const ClassInfo*> ks;
        for (auto& k : p.classes) ks.push_back(&k);
        launch_sort<T>(p, ks, std::vector<const void*>(ks.size(), p.d_x), kSortKeysToValues, false, st, launches,
                       nullptr, nullptr, false);
    }
    cudaEventRecord(p.t_setup1, st);
    LC_CK(cudaGetLastError());
    p.setup_done = true;
    return LC_OK;
}

// One amplitude-adjustment iteration of every class (Sec. 3.2.2).  Stage by
// stage over the classes: the transforms of the tile-path classes with one
// launch per kernel form and stage (launch_fft_iteration), those of the short
// classes per class, then the rank-order step of all of them with one launch
// per kernel form (launch_sort).  Classes touch disjoint parts of the plan's
// buffers, so their kernels of one stage can share a launch.
template <typename T>
static void enqueue_iteration(Plan& p, cudaStream_t st, uint64_t* launches, KernelTimes* kt = nullptr)
{
    // with the convergence test the FFTs work in d_f and d_keysB (free
    // until the sort starts) so that x_{i-1} stays in d_x for Eq. 4
    void* alt = p.conv_on ? p.d_keysB : p.d_x;
    std::vector<const ClassInfo*> tile, multi;
    for (auto& k : p.classes)
        if (!k.resident && k.log2n - 1 >= 12) tile.push_back(&k);
    if (kt) kt->begin(kGroupFFT, st);
    std::vector<void*> tile_out;
    if (!tile.empty()) launch_fft_iteration<T>(p, tile, p.d_x, p.d_f, alt, st, launches, tile_out);
    std::vector<const void*> src;
    size_t ti = 0;
    for (auto& k : p.classes) {
        if (k.resident) continue;
        void* R3;
        if (k.log2n - 1 >= 12) {
            // tile path: the spectral step runs inside the transforms' middle passes
            R3 = tile_out[ti++];
        } else {
            void* R1 = launch_fft<T>(p, k, false, p.d_x, p.d_f, nullptr, true, st, launches,
                                     p.conv_on ? p.d_keysB : nullptr);
            void* Zp = (R1 == p.d_f) ? alt : p.d_f;
            launch_spectral_iter<T>(p, k, R1, Zp, st);
            ++*launches;
            R3 = launch_fft<T>(p, k, true, Zp, R1, nullptr, true, st, launches);
        }
        multi.push_back(&k);
        src.push_back(R3);
    }
    if (kt) kt->end(st);
    if (!multi.empty()) {
        // the tile path's inverse transform has written the sample-sorted
        // classes' samples of x_adj (presampled)
        if (!p.conv_on) {
            launch_sort<T>(p, multi, src, kSortArgsortScatter, true, st, launches, nullptr, kt, true);
        } else {
            // the last sort pass reads keys A, so x_i can go to keys B; Eq. 4
            // then compares it with x_{i-1} in one coalesced pass
            launch_sort<T>(p, multi, src, kSortArgsortScatter, true, st, launches, p.d_keysB, kt, true);
            if (kt) kt->begin(kGroupOther, st);
            for (const ClassInfo* k : multi) {
                launch_conv_delta<T>(p, *k, p.d_keysB, st);
                launch_conv_finalize(p, *k, st);
                *launches += 2;
            }
            if (kt) kt->end(st);
        }
    }
    launch_iter_increment(p, st);
    ++*launches;
}

// Runs `n_it` more iterations.  reset: start from iteration 0 with every
// curve's budget = override_iters (or its job count); otherwise continue
// from the plan's current iteration index with the budgets already set.
template <typename T>
static lc_status run_iterations_impl(Plan& p, uint32_t override_iters, uint32_t n_it, bool reset,
                                     cudaStream_t st, uint64_t* launches)
{
    if (!p.setup_done) { set_error("lc_iterate before lc_setup/lc_generate"); return LC_ERR_INVALID; }
    cudaEventRecord(p.t_it0, st);
    if (reset) {
        launch_eff_iters(p, override_iters, st);
        ++*launches;
        if (p.conv_on) {
            launch_conv_reset(p, st);
            ++*launches;
        }
    }
    // curves of the fused on-chip classes run all n_it iterations in one launch
    for (auto& k : p.classes)
        if (k.resident && n_it > 0) launch_resident(p, k, n_it, st, launches);
    bool any_multi = false;
    for (auto& k : p.classes) any_multi |= !k.resident;
    if (any_multi && n_it > 0) {
        if (!p.iter_graph) {
            cudaGraph_t g = nullptr;
            uint64_t per = 0;
            LC_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            enqueue_iteration<T>(p, st, &per);
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(e)); return LC_ERR_CUDA; }
            e = cudaGraphInstantiate(&p.iter_graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { set_error(std::string("graph instantiate: ") + cudaGetErrorString(e)); return LC_ERR_CUDA; }
            p.launches_per_iter = per;
        }
        for (uint32_t it = 0; it < n_it; ++it) LC_CK(cudaGraphLaunch(p.iter_graph, st));
        *launches += (uint64_t)n_it * p.launches_per_iter;
    } else if (n_it > 0) {
        launch_iter_add(p, n_it, st);
        ++*launches;
    }
    cudaEventRecord(p.t_it1, st);
    p.timed_iter = true;
    LC_CK(cudaGetLastError());
    return LC_OK;
}

template <typename T>
static lc_status run_iterations(Plan& p, uint32_t override_iters, cudaStream_t st, uint64_t* launches)
{
    const uint32_t n_it = override_iters ? override_iters : p.max_iters;
    return run_iterations_impl<T>(p, override_iters, n_it, true, st, launches);
}

lc_status plan_setup(Plan& p, void* out_tk, cudaStream_t st, uint64_t* launches)
{
    return p.prec == LC_FP32 ? run_setup<float>(p, out_tk, st, launches) : run_setup<double>(p, out_tk, st, launches);
}

lc_status plan_continue(Plan& p, uint32_t n_it, cudaStream_t st, uint64_t* launches)
{
    return p.prec == LC_FP32 ? run_iterations_impl<float>(p, 0, n_it, false, st, launches)
                             : run_iterations_impl<double>(p, 0, n_it, false, st, launches);
}

void plan_free(Plan* p)
{
    if (!p) return;
    {
        DeviceGuard g(p->device);
        cudaStreamSynchronize(p->stream);
        if (p->iter_graph) cudaGraphExecDestroy(p->iter_graph);
        if (p->ext) {
            cudaFreeAsync(p->arena, p->stream);
            cudaStreamSynchronize(p->stream);
        } else {
            cudaFree(p->arena);
        }
        if (p->conv_arena) cudaFree(p->conv_arena);
        if (p->d_tk_stage) cudaFree(p->d_tk_stage);
        cudaEventDestroy(p->ev_in);
        cudaEventDestroy(p->ev_out);
        cudaEventDestroy(p->t_setup0);
        cudaEventDestroy(p->t_setup1);
        cudaEventDestroy(p->t_it0);
        cudaEventDestroy(p->t_it1);
        cudaStreamDestroy(p->stream);
    }
    delete p;
}

}  // namespace lc

using namespace lc;


extern "C" {

const char* lc_status_string(lc_status s)
{
    switch (s) {
    case LC_OK: return "LC_OK";
    case LC_PENDING: return "LC_PENDING";
    case LC_ERR_INVALID: return "LC_ERR_INVALID";
    case LC_ERR_NOMEM: return "LC_ERR_NOMEM";
    case LC_ERR_CUDA: return "LC_ERR_CUDA";
    case LC_ERR_TIMEOUT: return "LC_ERR_TIMEOUT";
    case LC_ERR_BUSY: return "LC_ERR_BUSY";
    case LC_ERR_UNKNOWN_TICKET: return "LC_ERR_UNKNOWN_TICKET";
    }
    return "LC_UNKNOWN_STATUS";
}

const char* lc_last_error(void) { return g_last_error.c_str(); }

lc_status lc_plan_create(const lc_job* jobs, size_t njobs, lc_precision prec, int device, lc_plan* out)
{
    if (!out) { set_error("out is null"); return LC_ERR_INVALID; }
    Plan* p = nullptr;
    lc_status s = plan_create(jobs, njobs, prec, device, &p);
    if (s != LC_OK) return s;
    *out = static_cast<lc_plan>(p);
    return LC_OK;
}

lc_status lc_plan_workspace_bytes(lc_plan plan, size_t* bytes)
{
    if (!plan || !bytes) { set_error("null argument"); return LC_ERR_INVALID; }
    *bytes = plan->arena_bytes;
    return LC_OK;
}

lc_status lc_plan_total_samples(lc_plan plan, size_t* samples)
{
    if (!plan || !samples) { set_error("null argument"); return LC_ERR_INVALID; }
    *samples = plan->total;
    return LC_OK;
}

lc_status lc_setup(lc_plan plan, void* out_tk, void* stream)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    uint64_t n = 0;
    lc_status s = plan->prec == LC_FP32 ? run_setup<float>(*plan, out_tk, plan->stream, &n)
                                        : run_setup<double>(*plan, out_tk, plan->stream, &n);
    plan->last_launches = n;
    return s;
}

lc_status lc_iterate(lc_plan plan, uint32_t iters, void* stream)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    if (!plan->setup_done) { set_error("lc_iterate before lc_setup/lc_generate"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    uint64_t n = 0;
    lc_status s = plan->prec == LC_FP32 ? run_iterations<float>(*plan, iters, plan->stream, &n)
                                        : run_iterations<double>(*plan, iters, plan->stream, &n);
    plan->last_launches = n;
    return s;
}

lc_status lc_generate(lc_plan plan, void* out_x, void* out_tk, void* stream)
{
    if (!plan || !out_x) { set_error("null plan or out_x"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    uint64_t n = 0;
    lc_status s = plan->prec == LC_FP32 ? run_setup<float>(*plan, out_tk, plan->stream, &n)
                                        : run_setup<double>(*plan, out_tk, plan->stream, &n);
    if (s == LC_OK)
        s = plan->prec == LC_FP32 ? run_iterations<float>(*plan, 0, plan->stream, &n)
                                  : run_iterations<double>(*plan, 0, plan->stream, &n);
    if (s == LC_OK) {
        const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
        LC_CK(cudaMemcpyAsync(out_x, plan->d_x, plan->total * ts, cudaMemcpyDeviceToDevice, plan->stream));
    }
    plan->last_launches = n;
    return s;
}

lc_status lc_generate_host(lc_plan plan, void* out_x_host, void* out_tk_host, void* stream)
{
    if (!plan || !out_x_host) { set_error("null plan or out_x_host"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
    if (out_tk_host && !plan->d_tk_stage) {
        if (cudaMalloc(&plan->d_tk_stage, plan->total * ts) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of the TK95 staging buffer failed");
            return LC_ERR_NOMEM;
        }
    }
    uint64_t n = 0;
    lc_status s;
    {
        StreamJoin j(*plan, stream);
        void* tk = out_tk_host ? plan->d_tk_stage : nullptr;
        s = plan->prec == LC_FP32 ? run_setup<float>(*plan, tk, plan->stream, &n)
                                  : run_setup<double>(*plan, tk, plan->stream, &n);
        if (s == LC_OK && out_tk_host)
            LC_CK(cudaMemcpyAsync(out_tk_host, tk, plan->total * ts, cudaMemcpyDeviceToHost, plan->stream));
        if (s == LC_OK)
            s = plan->prec == LC_FP32 ? run_iterations<float>(*plan, 0, plan->stream, &n)
                                      : run_iterations<double>(*plan, 0, plan->stream, &n);
        if (s == LC_OK)
            LC_CK(cudaMemcpyAsync(out_x_host, plan->d_x, plan->total * ts, cudaMemcpyDeviceToHost, plan->stream));
    }
    plan->last_launches = n;
    if (s != LC_OK) return s;
    LC_CK(cudaStreamSynchronize(plan->stream));
    return LC_OK;
}

lc_status lc_get_state(lc_plan plan, void* out_x, void* stream)
{
    if (!plan || !out_x) { set_error("null argument"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
    LC_CK(cudaMemcpyAsync(out_x, plan->d_x, plan->total * ts, cudaMemcpyDeviceToDevice, plan->stream));
    return LC_OK;
}

lc_status lc_set_state(lc_plan plan, const void* in_x, void* stream)
{
    if (!plan || !in_x) { set_error("null argument"); return LC_ERR_INVALID; }
    if (!plan->setup_done) { set_error("lc_set_state before lc_setup/lc_generate"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
    LC_CK(cudaMemcpyAsync(plan->d_x, in_x, plan->total * ts, cudaMemcpyDeviceToDevice, plan->stream));
    return LC_OK;
}

lc_status lc_rank_replace(lc_plan plan, const void* x_adj, void* out_x, void* stream)
{
    if (!plan || !x_adj || !out_x) { set_error("null argument"); return LC_ERR_INVALID; }
    if (!plan->setup_done) { set_error("lc_rank_replace before lc_setup/lc_generate"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
    // the sort reads its values from the FFT buffer, as in an iteration
    LC_CK(cudaMemcpyAsync(plan->d_f, x_adj, plan->total * ts, cudaMemcpyDeviceToDevice, plan->stream));
    uint64_t n = 0;
    for (auto& k : plan->classes) {
        if (plan->prec == LC_FP32)
            launch_sort<float>(*plan, k, plan->d_f, kSortArgsortScatter, false, plan->stream, &n, out_x);
        else
            launch_sort<double>(*plan, k, plan->d_f, kSortArgsortScatter, false, plan->stream, &n, out_x);
    }
    plan->last_launches = n + 1;
    LC_CK(cudaGetLastError());
    return LC_OK;
}

lc_status lc_plan_buffer(lc_plan plan, int which, const void** device_ptr, size_t* bytes)
{
    if (!plan || !device_ptr) { set_error("null argument"); return LC_ERR_INVALID; }
    const size_t ts = plan->prec == LC_FP32 ? 4 : 8;
    switch (which) {
    case 0: *device_ptr = plan->d_x; if (bytes) *bytes = plan->total * ts; return LC_OK;
    case 1: *device_ptr = plan->d_A; if (bytes) *bytes = plan->total_h * ts; return LC_OK;
    case 2: *device_ptr = plan->d_s; if (bytes) *bytes = plan->total * ts; return LC_OK;
    default: set_error("which must be 0, 1 or 2"); return LC_ERR_INVALID;
    }
}

lc_status lc_plan_last_launches(lc_plan plan, uint64_t* launches)
{
    if (!plan || !launches) { set_error("null argument"); return LC_ERR_INVALID; }
    *launches = plan->last_launches;
    return LC_OK;
}

lc_status lc_plan_timing(lc_plan plan, float* setup_ms, float* iterate_ms)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    float a = 0.f, b = 0.f;
    if (plan->timed_setup) {
        LC_CK(cudaEventSynchronize(plan->t_setup1));
        LC_CK(cudaEventElapsedTime(&a, plan->t_setup0, plan->t_setup1));
    }
    if (plan->timed_iter) {
        LC_CK(cudaEventSynchronize(plan->t_it1));
        LC_CK(cudaEventElapsedTime(&b, plan->t_it0, plan->t_it1));
    }
    if (setup_ms) *setup_ms = a;
    if (iterate_ms) *iterate_ms = b;
    return LC_OK;
}

lc_status lc_plan_set_convergence(lc_plan plan, const double* thresholds, uint32_t history)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    if (history < 1 || history > (1u << 16)) { set_error("history must be in [1, 65536]"); return LC_ERR_INVALID; }
    const size_t nc = plan->ncurves;
    std::vector<double> thr(nc, 0.0);
    for (size_t c = 0; c < nc; ++c) {
        if (thresholds) {
            if (std::isnan(thresholds[c])) { set_error("threshold " + std::to_string(c) + " is NaN"); return LC_ERR_INVALID; }
            thr[c] = thresholds[c];
        }
        // Eq. 4 takes logs of the values: float draws must stay normal numbers
        if (plan->prec == LC_FP32 && plan->jobs[c].erdf.log_lmin < -37.0) {
            set_error("job " + std::to_string(c) + ": log_lmin below -37 gives FP32 values below FLT_MIN");
            return LC_ERR_INVALID;
        }
    }
    DeviceGuard g(plan->device);
    LC_CK(cudaStreamSynchronize(plan->stream));
    size_t part = 0;
    for (auto& k : plan->classes) {
        const int C = k.resident && k.log2n > 14 ? 1 << (k.log2n - 14) : 0;
        part = std::max(part, (size_t)k.ncurves * (size_t)std::max(k.tiles_per_curve, C));
    }
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_thr = up(nc * 8), b_delta = up(nc * (size_t)history * 8), b_part = up(part * 8);
    if (plan->conv_arena && (plan->conv.hist != history || plan->conv_part != part)) {
        cudaFree(plan->conv_arena);
        plan->conv_arena = nullptr;
    }
    if (!plan->conv_arena) {
        if (cudaMalloc(&plan->conv_arena, b_thr + b_delta + b_part) != cudaSuccess) {
            cudaGetLastError();
            plan->conv_on = false;
            set_error("device allocation of the convergence record failed");
            return LC_ERR_NOMEM;
        }
    }
    char* b = (char*)plan->conv_arena;
    plan->conv.thr = (const double*)b;
    plan->conv.delta = (double*)(b + b_thr);
    plan->conv.part = (double*)(b + b_thr + b_delta);
    plan->conv.hist = history;
    plan->conv_part = part;
    plan->conv_on = true;
    LC_CK(cudaMemcpyAsync((void*)plan->conv.thr, thr.data(), nc * 8, cudaMemcpyHostToDevice, plan->stream));
    launch_conv_reset(*plan, plan->stream);
    LC_CK(cudaStreamSynchronize(plan->stream));
    // the captured iteration graph has the kernels of the other mode
    if (plan->iter_graph) {
        cudaGraphExecDestroy(plan->iter_graph);
        plan->iter_graph = nullptr;
    }
    return LC_OK;
}

lc_status lc_plan_convergence(lc_plan plan, double* deltas, uint32_t* iters_run)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    if (!plan->conv_on) { set_error("lc_plan_convergence before lc_plan_set_convergence"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    LC_CK(cudaStreamSynchronize(plan->stream));
    const size_t nc = plan->ncurves;
    std::vector<uint32_t> eff(nc);
    int it = 0;
    if (deltas)
        LC_CK(cudaMemcpyAsync(deltas, plan->conv.delta, nc * (size_t)plan->conv.hist * 8, cudaMemcpyDeviceToHost,
                              plan->stream));
    LC_CK(cudaMemcpyAsync(eff.data(), plan->d_eff_iters, nc * 4, cudaMemcpyDeviceToHost, plan->stream));
    LC_CK(cudaMemcpyAsync(&it, plan->d_iter, sizeof(int), cudaMemcpyDeviceToHost, plan->stream));
    LC_CK(cudaStreamSynchronize(plan->stream));
    if (iters_run)
        for (size_t c = 0; c < nc; ++c) iters_run[c] = std::min(eff[c], (uint32_t)std::max(it, 0));
    return LC_OK;
}

lc_status lc_plan_profile(lc_plan plan, float* group_ms, size_t ngroups, uint64_t* counts)
{
    if (!plan || !group_ms) { set_error("null plan or group_ms"); return LC_ERR_INVALID; }
    if (!plan->setup_done) { set_error("lc_plan_profile before lc_setup/lc_generate"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    Plan& p = *plan;
    cudaStream_t st = p.stream;
    LC_CK(cudaStreamSynchronize(st));
    uint64_t launches = 0;
    {
        KernelTimes kt;
        launch_eff_iters(p, 1, st);  // one iteration of every curve, counter from 0
        for (auto& k : p.classes) {
            if (!k.resident) continue;
            kt.begin(kGroupResident, st);
            launch_resident(p, k, 1, st, &launches);
            kt.end(st);
        }
        if (p.prec == LC_FP32) enqueue_iteration<float>(p, st, &launches, &kt);
        else enqueue_iteration<double>(p, st, &launches, &kt);
        LC_CK(cudaGetLastError());
        LC_CK(cudaStreamSynchronize(st));
        std::vector<float> sums(kGroups, 0.f);
        uint64_t nscatter = 0;
        for (auto& s : kt.spans) {
            float ms = 0.f;
            LC_CK(cudaEventElapsedTime(&ms, s.a, s.b));
            sums[s.group] += ms;
            nscatter += s.group == kGroupSortScatter;
        }
        for (size_t q = 0; q < ngroups; ++q) group_ms[q] = q < (size_t)kGroups ? sums[q] : 0.f;
        if (counts) counts[0] = nscatter;
    }
    if (counts) {
        uint64_t multi = 0, fused = 0, bucket = 0;
        for (auto& k : p.classes) {
            (k.resident ? fused : multi) += (uint64_t)k.ncurves << k.log2n;
            if (!k.resident && k.bucket) bucket += (uint64_t)k.ncurves << k.log2n;
        }
        counts[1] = multi;
        counts[2] = fused;
        counts[3] = bucket;
    }
    p.timed_iter = false;
    return LC_OK;
}

lc_status lc_plan_destroy(lc_plan plan)
{
    if (!plan) { set_error("null plan"); return LC_ERR_INVALID; }
    plan_free(static_cast<Plan*>(plan));
    return LC_OK;
}

}  // extern "C"

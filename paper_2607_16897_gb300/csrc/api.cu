// C ABI of libglt.so (declared in include/glt.h): argument checking, device
// memory ownership, stream ordering, and the batch / CUDA-graph / autotuner
// plumbing around the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "glt_internal.h"

namespace glt {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return GLT_ERR_CUDA;
}

static int invalid(const char* msg)
{
    set_error(msg);
    return GLT_ERR_INVALID_ARG;
}

#define GLT_CHECK(call, what)                               \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// A batch's launch classes (see glt_batch) and, for the autotuner, their time.
struct ClassTable {
    int nclass = 1;
    int first[kMaxBatchClasses + 1] = {};
    int cluster[kMaxBatchClasses] = {};
    int threads[kMaxBatchClasses] = {};
    float ms = 0.0f;
};
// Autotuner results of this process, keyed by the batch signature.
using TuneResult = ClassTable;

static void apply_table(glt_batch* b, const ClassTable& c)
{
    b->nclass = c.nclass;
    for (int k = 0; k <= c.nclass; ++k) b->cls_first[k] = c.first[k];
    for (int k = 0; k < c.nclass; ++k) {
        b->cls_cluster[k] = c.cluster[k];
        b->cls_threads[k] = c.threads[k];
    }
}

static ClassTable uniform_table(int S, int cluster, int threads)
{
    ClassTable c;
    c.nclass = 1;
    c.first[0] = 0;
    c.first[1] = S;
    c.cluster[0] = cluster;
    c.threads[0] = threads;
    return c;
}

static void set_uniform(glt_batch* b, int cluster, int threads)
{
    apply_table(b, uniform_table(b->S, cluster, threads));
}

// Two classes: the first `heavy` streams of the launch order and the rest
// (one class when heavy is 0 or S).
static ClassTable split_table(int S, int heavy, int hc, int ht, int lc, int lt)
{
    if (heavy >= S) return uniform_table(S, hc, ht);
    if (heavy <= 0) return uniform_table(S, lc, lt);
    ClassTable c;
    c.nclass = 2;
    c.first[0] = 0;
    c.first[1] = heavy;
    c.first[2] = S;
    c.cluster[0] = hc;
    c.threads[0] = ht;
    c.cluster[1] = lc;
    c.threads[1] = lt;
    return c;
}

// Clusters in proportion to work: stream i of the launch order gets the
// smallest power-of-two cluster c <= 16 with c * points_per_cta >= its point
// capacity in 8-sample units (max_points * K / 8), reduced to the largest
// size that can launch with `threads`; streams of equal c form a class.  The
// launch order is by descending capacity x K, so c never grows along it and
// the classes are contiguous ranges (at most one per size).  False if no
// cluster size can launch with `threads`.
static bool proportional_table(const glt_batch* b, int points_per_cta, int threads, ClassTable& c)
{
    c = ClassTable{};
    c.nclass = 0;
    int prev = 0;
    for (int i = 0; i < b->S; ++i) {
        const glt_tracker* t = b->trk[b->order[i]];
        const long long work = (long long)t->cfg.max_points * t->K / 8;
        int cl = 1;
        while (cl < 16 && (long long)cl * points_per_cta < work) cl *= 2;
        while (cl > 1 && !track_shape_ok(cl, threads, b->variant)) cl /= 2;
        if (!track_shape_ok(cl, threads, b->variant)) return false;
        if (cl != prev) {
            if (c.nclass == kMaxBatchClasses) return false;
            c.first[c.nclass] = i;
            c.cluster[c.nclass] = cl;
            c.threads[c.nclass] = threads;
            ++c.nclass;
            prev = cl;
        }
    }
    c.first[c.nclass] = b->S;
    return c.nclass > 0;
}
static std::mutex g_tune_mutex;
static std::map<std::string, TuneResult> g_tune_cache;

static void set_identity(double T[12])
{
    for (int i = 0; i < 12; ++i) T[i] = (i % 5 == 0) ? 1.0 : 0.0;   // entries 0, 5, 10
}

static void reset_state_pose(glt_state& st)
{
    set_identity(st.T_cr);
    st.a = 0.0;
    st.b = 0.0;
    st.frames = 0;
}

static bool finite_all(const double* v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

template <class T>
static cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

static void free_tracker(glt_tracker* t)
{
    if (!t) return;
    for (int s = 0; s < 2; ++s) cudaFree(t->pyr[s].base);
    cudaFree(t->packed);
    cudaFree(t->uvd_dev);
    cudaFree(t->pt);
    cudaFree(t->dz);
    cudaFree(t->I0);
    cudaFree(t->G0);
    cudaFree(t->Hc);
    cudaFree(t->desc_dev);
    cudaFree(t->desc_ptr_dev);
    cudaFree(t->user_dev);
    cudaFree(t->trace_count);
    cudaFree(t->jobs_dev);
    cudaFree(t->pack_dev);
    cudaFree(t->init_dev);
    cudaFree(t->result_dev);
    cudaFree(t->trace_E);
    cudaFree(t->trace_n);
    cudaFree(t->trace_info);
    cudaFree(t->lin_partials);
    cudaFree(t->lin_counter);
    cudaFree(t->lin_out);
    cudaFree(t->lin_res);
    cudaFree(t->stage_dev);
    cudaFreeHost(t->h_init);
    cudaFreeHost(t->h_result);
    cudaFreeHost(t->h_lin);
    delete t;
}

static int check_config(const glt_config* c)
{
    if (!c) return invalid("config is NULL");
    if (c->width < 16 || c->height < 16 || c->width > (1 << 15) || c->height > (1 << 15))
        return invalid("width/height must be in [16, 32768]");
    if (c->levels < 1 || c->levels > GLT_MAX_LEVELS) return invalid("levels must be in [1, 8]");
    if ((c->width >> (c->levels - 1)) < 8 || (c->height >> (c->levels - 1)) < 8)
        return invalid("the coarsest level must be at least 8 x 8 pixels");
    if (!(c->fx > 0 && c->fy > 0) || !std::isfinite(c->fx) || !std::isfinite(c->fy) ||
        !std::isfinite(c->cx) || !std::isfinite(c->cy))
        return invalid("intrinsics must be finite with fx, fy > 0");
    if (c->max_points < 1 || c->max_points > (1 << 22)) return invalid("max_points must be in [1, 4194304]");
    for (int l = 0; l < c->levels; ++l)
        if (c->max_iters[l] < 0 || c->max_iters[l] > 1000) return invalid("max_iters must be in [0, 1000]");
    if (!(c->huber_k > 0) || !std::isfinite(c->huber_k)) return invalid("huber_k must be > 0");
    if (!(c->lambda0 >= 0) || !std::isfinite(c->lambda0) || !(c->lambda_up >= 1) || !(c->lambda_down > 0) || !(c->lambda_down <= 1))
        return invalid("LM damping factors out of range");
    if (!(c->eps_step >= 0) || !(c->eps_step_coarse >= 0) || !(c->eps_cost >= 0) ||
        !(c->accept_step >= 0))
        return invalid("eps_step / eps_step_coarse / eps_cost / accept_step must be >= 0");
    if (c->min_valid < 1) return invalid("min_valid must be >= 1");
    if (!(c->zmin > 0)) return invalid("zmin must be > 0");
    if (c->precision != GLT_FP32 && c->precision != GLT_MIXED) return invalid("unknown precision");
    if (c->cluster < 0 || c->cluster > 16) return invalid("cluster must be in [0, 16]");
    if (c->threads != 0 && c->threads != 128 && c->threads != 256 && c->threads != 512)
        return invalid("threads must be 0, 128, 256 or 512");
    if (c->jacobian != GLT_FORWARD && c->jacobian != GLT_IC)
        return invalid("jacobian must be GLT_FORWARD or GLT_IC");
    if (c->pattern != 0 && (c->pattern < 3 || c->pattern > 11 || (c->pattern & 1) == 0))
        return invalid("pattern must be 0 (8-pixel) or an odd patch size 3..11");
    if (c->pattern != 0 && c->precision != GLT_FP32)
        return invalid("p x p patches need precision GLT_FP32");
    if (c->affine != 0 && c->affine != 1) return invalid("affine must be 0 or 1");
    if (c->hessian != GLT_HESSIAN_PASS && c->hessian != GLT_HESSIAN_CACHED)
        return invalid("hessian must be GLT_HESSIAN_PASS or GLT_HESSIAN_CACHED");
    if (c->solve != GLT_SOLVE_FP64 && c->solve != GLT_SOLVE_FP32)
        return invalid("solve must be GLT_SOLVE_FP64 or GLT_SOLVE_FP32");
    if (c->hessian == GLT_HESSIAN_CACHED &&
        (c->jacobian != GLT_IC || c->affine != 0 || c->lambda0 != 0.0 || c->precision != GLT_FP32 ||
         (c->threads != 0 && c->threads != 512)))
        return invalid("GLT_HESSIAN_CACHED needs jacobian GLT_IC, affine 0, lambda0 0, "
                       "precision GLT_FP32 and 512 (or 0) threads");
    if (c->hessian != GLT_HESSIAN_CACHED && c->pattern != 0 && c->threads != 0 && c->threads != 256)
        return invalid("p x p patches run with 256 threads per CTA");
    return GLT_OK;
}

// CTAs per stream for n points when the caller left it to the library.
static void resolve_shape(glt_tracker* t)
{
    const int variant = track_variant(t->cfg);
    int threads = t->cfg.threads ? t->cfg.threads : (variant == 4 ? 512 : 256);
    int cluster = t->cfg.cluster;
    if (cluster == 0) {
        // about one point per thread, in units of the 8-pixel pattern's work
        // (the cached-Hessian form: one task per thread)
        const long long work = variant == 4 ? (long long)t->N * hc_groups(t->cfg.pattern)
                                            : (long long)t->N * std::max(1, t->K / 8);
        cluster = (int)std::min<long long>(16, std::max<long long>(1, (work + threads - 1) / threads));
    }
    while (cluster > 1 && !track_shape_ok(cluster, threads, variant)) cluster = cluster > 8 ? 8 : cluster - 1;
    t->cluster = cluster;
    t->threads = threads;
}

}  // namespace glt

using namespace glt;

extern "C" {

const char* glt_status_string(int code)
{
    switch (code) {
    case GLT_OK: return "ok";
    case GLT_ERR_INVALID_ARG: return "invalid argument";
    case GLT_ERR_CUDA: return "CUDA error";
    case GLT_ERR_NO_REFERENCE: return "no reference";
    case GLT_ERR_CAPACITY: return "capacity exceeded";
    case GLT_ERR_UNSUPPORTED: return "unsupported";
    case GLT_ERR_IO: return "file error";
    default: break;
    }
    // status bits: every combination of the four per-frame outcomes
    static const char* const kBits[16] = {
        "ok", "too few points", "not positive definite", "too few points|not positive definite",
        "diverged", "too few points|diverged", "not positive definite|diverged",
        "too few points|not positive definite|diverged", "timeout", "too few points|timeout",
        "not positive definite|timeout", "too few points|not positive definite|timeout",
        "diverged|timeout", "too few points|diverged|timeout", "not positive definite|diverged|timeout",
        "too few points|not positive definite|diverged|timeout"};
    if (code > 0 && code < 16) return kBits[code];
    return "unknown";
}

const char* glt_last_error(void) { return g_err.c_str(); }

const char* glt_version(void) { return "glt 0.1 (sm_103a)"; }

void glt_default_config(glt_config* c, int width, int height, double fx, double fy, double cx,
                        double cy)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->width = width;
    c->height = height;
    c->levels = 4;
    c->fx = fx;
    c->fy = fy;
    c->cx = cx;
    c->cy = cy;
    c->max_points = 4096;
    for (int l = 0; l < GLT_MAX_LEVELS; ++l) c->max_iters[l] = 10;
    c->huber_k = 9.0;
    c->lambda0 = 1e-4;
    c->lambda_up = 4.0;
    c->lambda_down = 0.5;
    c->eps_step = 1e-6;
    c->eps_step_coarse = 3e-4;
    c->eps_cost = 0.0;
    c->accept_step = 1e-3;
    c->min_valid = 16;
    c->zmin = 1e-3;
    c->precision = GLT_FP32;
    c->cluster = 0;
    c->threads = 0;
    c->jacobian = GLT_FORWARD;
    c->pattern = 0;
    c->affine = 1;
    c->hessian = GLT_HESSIAN_PASS;
    c->solve = GLT_SOLVE_FP64;
}

int glt_create(const glt_config* cfg, glt_tracker** out)
{
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc != GLT_OK) return rc;
    glt_tracker* t = new glt_tracker();
    t->cfg = *cfg;
    t->L = cfg->levels;
    reset_state_pose(t->state);
    set_identity(t->state.motion);
    cudaError_t e = cudaGetDevice(&t->device);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "cudaGetDevice");
    }
#define ALLOC(call)                                 \
    do {                                            \
        cudaError_t e2 = (call);                    \
        if (e2 != cudaSuccess) {                    \
            free_tracker(t);                        \
            return cuda_fail(e2, "device allocation"); \
        }                                           \
    } while (0)
    size_t pix = 0;
    for (int l = 0; l < t->L; ++l) {
        t->W[l] = cfg->width >> l;
        t->H[l] = cfg->height >> l;
        t->pitch[l] = (int)align_up((size_t)t->W[l] + 8, 16);
        t->poff[l] = pix;
        pix += (size_t)t->W[l] * t->H[l];
    }
    for (int s = 0; s < 2; ++s) {
        size_t off = 0;
        for (int l = 0; l < t->L; ++l) {
            t->pyr[s].off[l] = off;
            off = align_up(off + (size_t)t->pitch[l] * t->H[l], 256);
        }
        t->pyr[s].bytes = off + 256;
        ALLOC(dalloc(&t->pyr[s].base, t->pyr[s].bytes));
        ALLOC(cudaMemset(t->pyr[s].base, 0, t->pyr[s].bytes));
    }
    if (cfg->precision == GLT_MIXED) ALLOC(dalloc(&t->packed, pix));
    const int maxp = cfg->max_points;
    t->Npad = (int)align_up((size_t)maxp, 32);
    ALLOC(dalloc(&t->uvd_dev, (size_t)maxp * 3));
    ALLOC(dalloc(&t->pt, (size_t)t->Npad));
    ALLOC(dalloc(&t->dz, (size_t)t->Npad));
    t->K = cfg->pattern == 0 ? 8 : cfg->pattern * cfg->pattern;
    ALLOC(dalloc(&t->I0, (size_t)t->L * t->Npad * t->K));
    if (cfg->jacobian == GLT_IC) ALLOC(dalloc(&t->G0, (size_t)t->L * t->Npad * t->K));
    if (cfg->hessian == GLT_HESSIAN_CACHED) ALLOC(dalloc(&t->Hc, (size_t)t->L * 72));
    ALLOC(dalloc(&t->desc_dev, 1));
    ALLOC(dalloc(&t->desc_ptr_dev, 1));
    ALLOC(dalloc(&t->user_dev, 1));
    ALLOC(dalloc(&t->trace_count, 1));
    ALLOC(dalloc(&t->jobs_dev, (size_t)2 * GLT_MAX_LEVELS));
    ALLOC(dalloc(&t->pack_dev, (size_t)GLT_MAX_LEVELS));
    ALLOC(dalloc(&t->init_dev, 14));
    ALLOC(dalloc(&t->result_dev, 1));
    int maxit = 0;
    for (int l = 0; l < t->L; ++l) maxit = std::max(maxit, cfg->max_iters[l]);
    t->max_trace = t->L * (1 + maxit);
    ALLOC(dalloc(&t->trace_E, (size_t)t->max_trace));
    ALLOC(dalloc(&t->trace_n, (size_t)t->max_trace));
    ALLOC(dalloc(&t->trace_info, (size_t)t->max_trace));
    t->lin_blocks = (maxp + 127) / 128;
    ALLOC(dalloc(&t->lin_partials, (size_t)t->lin_blocks * kAccPad));
    ALLOC(dalloc(&t->lin_counter, 1));
    ALLOC(cudaMemset(t->lin_counter, 0, sizeof(unsigned)));
    ALLOC(dalloc(&t->lin_out, (size_t)kAccPad));
    ALLOC(dalloc(&t->lin_res, (size_t)maxp * t->K));
    ALLOC(dalloc(&t->stage_dev, (size_t)t->W[0] * t->H[0]));
    ALLOC(cudaMallocHost(reinterpret_cast<void**>(&t->h_init), 14 * sizeof(double)));
    ALLOC(cudaMallocHost(reinterpret_cast<void**>(&t->h_result), sizeof(glt_result)));
    ALLOC(cudaMallocHost(reinterpret_cast<void**>(&t->h_lin), kAccPad * sizeof(double)));

    // descriptor
    StreamDesc& D = t->desc_host;
    std::memset(&D, 0, sizeof(D));
    for (int l = 0; l < t->L; ++l) {
        D.lv[l].img = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l];
        D.lv[l].packed = t->packed ? t->packed + t->poff[l] : nullptr;
        D.lv[l].W = t->W[l];
        D.lv[l].H = t->H[l];
        D.lv[l].pitch = t->pitch[l];
    }
    D.L = t->L;
    D.N = 0;
    D.Npad = t->Npad;
    D.fx = (float)cfg->fx;
    D.fy = (float)cfg->fy;
    D.huber_k = (float)cfg->huber_k;
    D.zmin = (float)cfg->zmin;
    D.pt = t->pt;
    D.dz = t->dz;
    D.I0 = t->I0;
    D.G0 = t->G0;
    D.Hc = t->Hc;
    D.solve = t->cfg.solve;
    D.pattern = cfg->pattern;
    D.K = t->K;
    D.affine = cfg->affine;
    for (int l = 0; l < GLT_MAX_LEVELS; ++l) D.max_iters[l] = l < t->L ? cfg->max_iters[l] : 0;
    D.min_valid = cfg->min_valid;
    D.max_trace = t->max_trace;
    D.lambda0 = cfg->lambda0;
    D.lambda_up = cfg->lambda_up;
    D.lambda_down = cfg->lambda_down;
    D.eps_step = cfg->eps_step;
    D.eps_step_coarse = cfg->eps_step_coarse;
    D.eps_cost = cfg->eps_cost;
    D.accept_step = cfg->accept_step;
    D.trace_E = t->trace_E;
    D.trace_n = t->trace_n;
    D.trace_info = t->trace_info;
    D.trace_count = t->trace_count;
    ALLOC(cudaMemcpy(t->desc_dev, &D, sizeof(D), cudaMemcpyHostToDevice));
    ALLOC(cudaMemcpy(t->desc_ptr_dev, &t->desc_dev, sizeof(StreamDesc*), cudaMemcpyHostToDevice));
    const int zero = 0;
    ALLOC(cudaMemcpy(t->user_dev, &zero, sizeof(int), cudaMemcpyHostToDevice));
    ALLOC(cudaMemcpy(t->trace_count, &zero, sizeof(int), cudaMemcpyHostToDevice));

    // pyramid jobs per slot: level l-1 -> l
    std::vector<PyrJob> jobs(2 * GLT_MAX_LEVELS);
    for (int s = 0; s < 2; ++s)
        for (int l = 1; l < t->L; ++l) {
            PyrJob& J = jobs[s * GLT_MAX_LEVELS + (l - 1)];
            J.src = t->pyr[s].base + t->pyr[s].off[l - 1];
            J.dst = t->pyr[s].base + t->pyr[s].off[l];
            J.sW = t->W[l - 1];
            J.sH = t->H[l - 1];
            J.sp = t->pitch[l - 1];
            J.dW = t->W[l];
            J.dH = t->H[l];
            J.dp = t->pitch[l];
        }
    ALLOC(cudaMemcpy(t->jobs_dev, jobs.data(), jobs.size() * sizeof(PyrJob), cudaMemcpyHostToDevice));
    std::vector<PackJob> packs(GLT_MAX_LEVELS);
    for (int l = 0; l < t->L; ++l) {
        packs[l].src = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l];
        packs[l].dst = t->packed ? t->packed + t->poff[l] : nullptr;
        packs[l].W = t->packed ? t->W[l] : 0;
        packs[l].H = t->H[l];
        packs[l].sp = t->pitch[l];
    }
    ALLOC(cudaMemcpy(t->pack_dev, packs.data(), packs.size() * sizeof(PackJob), cudaMemcpyHostToDevice));
#undef ALLOC
    resolve_shape(t);
    *out = t;
    return GLT_OK;
}

void glt_destroy(glt_tracker* trk) { free_tracker(trk); }

int glt_build_pyramid(glt_tracker* t, int slot, const uint8_t* img, int pitch_bytes, int is_device,
                      void* stream)
{
    if (!t || !img) return invalid("tracker or image is NULL");
    if (slot != GLT_REF && slot != GLT_CUR) return invalid("slot must be GLT_REF or GLT_CUR");
    if (pitch_bytes < t->cfg.width) return invalid("pitch_bytes < width");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Pyramid& P = t->pyr[slot];
    if (!is_device && t->L > 1) {
        // host frame: one copy into the tracker's device staging buffer, then
        // the device path (level 1 reads it and writes level 0)
        const size_t W = (size_t)t->W[0], H = (size_t)t->H[0];
        if ((size_t)pitch_bytes == W)
            GLT_CHECK(cudaMemcpyAsync(t->stage_dev, img, W * H, cudaMemcpyHostToDevice, s), "frame upload");
        else
            GLT_CHECK(cudaMemcpy2DAsync(t->stage_dev, W, img, (size_t)pitch_bytes, W, H,
                                        cudaMemcpyHostToDevice, s),
                      "frame upload");
        img = t->stage_dev;
        pitch_bytes = (int)W;
        is_device = 1;
    }
    // every kernel after the first is a programmatic dependent of the one
    // before it (it starts early and waits on the device for its source level)
    if (is_device && t->L > 1) {
        // level 1 straight from the caller's frame; its tiles write level 0
        for (int l = 1; l < t->L; ++l)
            GLT_CHECK(launch_pyr_down(t->jobs_dev + slot * GLT_MAX_LEVELS + (l - 1), nullptr,
                                      pyr_tiles_x(t->W[l]) * pyr_tiles_y(t->H[l]), s, nullptr,
                                      l == 1 ? img : nullptr, l == 1 ? pitch_bytes : 0, l > 1),
                      "pyramid kernel");
        if (slot == GLT_CUR && t->packed)
            GLT_CHECK(launch_pack(t->pack_dev, t->L, t->W[0] * t->H[0], s, true), "pack kernel");
        P.built = true;
        return GLT_OK;
    }
    GLT_CHECK(cudaMemcpy2DAsync(P.base + P.off[0], (size_t)t->pitch[0], img, (size_t)pitch_bytes,
                                (size_t)t->W[0], (size_t)t->H[0],
                                is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
              "level-0 copy");
    for (int l = 1; l < t->L; ++l)
        GLT_CHECK(launch_pyr_down(t->jobs_dev + slot * GLT_MAX_LEVELS + (l - 1), nullptr,
                                  pyr_tiles_x(t->W[l]) * pyr_tiles_y(t->H[l]), s, nullptr, nullptr, 0,
                                  l > 1),
                  "pyramid kernel");
    if (slot == GLT_CUR && t->packed) {
        GLT_CHECK(launch_pack(t->pack_dev, t->L, t->W[0] * t->H[0], s, t->L > 1), "pack kernel");
    }
    P.built = true;
    return GLT_OK;
}

int glt_set_map_points(glt_tracker* t, const float* uvd, int n, int is_device, void* stream)
{
    if (!t) return invalid("tracker is NULL");
    if (n < 0 || (n > 0 && !uvd)) return invalid("bad point array");
    if (n > t->cfg.max_points) {
        set_error("more map points than max_points");
        return GLT_ERR_CAPACITY;
    }
    if (!t->pyr[GLT_REF].built) {
        set_error("glt_build_pyramid(GLT_REF) must come first");
        return GLT_ERR_NO_REFERENCE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float* src = uvd;
    if (n > 0 && !is_device) {
        GLT_CHECK(cudaMemcpyAsync(t->uvd_dev, uvd, (size_t)n * 3 * sizeof(float),
                                  cudaMemcpyHostToDevice, s),
                  "map point upload");
        src = t->uvd_dev;
    }
    const bool n_changed = t->N != n || !t->have_points;
    t->N = n;
    t->desc_host.N = n;
    // the kernel also stores n into the device descriptor (no host upload)
    GLT_CHECK(launch_set_points(t, src, n, s), "map point kernel");
    if (t->Hc) GLT_CHECK(launch_ic_hessian(t, s), "reference Hessian kernel");
    t->have_points = true;
    t->version++;
    // a new reference: the state's pose restarts at the reference (motion kept)
    reset_state_pose(t->state);
    t->state.reference = t->version;
    if (n_changed) resolve_shape(t);
    return GLT_OK;
}

static int track_prereq(glt_tracker* t)
{
    if (!t) return invalid("tracker is NULL");
    if (!t->have_points) {
        set_error("glt_set_map_points must come first");
        return GLT_ERR_NO_REFERENCE;
    }
    if (!t->pyr[GLT_CUR].built) return invalid("glt_build_pyramid(GLT_CUR) must come first");
    return GLT_OK;
}

int glt_track_frame_async(glt_tracker* t, const double* init_dev, glt_result* out_dev, void* stream)
{
    int rc = track_prereq(t);
    if (rc != GLT_OK) return rc;
    if (!init_dev || !out_dev) return invalid("init_dev / out_dev is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    GLT_CHECK(launch_track(t->desc_ptr_dev, t->user_dev, 1, t->cluster, t->threads,
                           track_variant(t->cfg), init_dev, out_dev, s),
              "track kernel");
    return GLT_OK;
}

int glt_track_image_async(glt_tracker* t, const uint8_t* frame_dev, int pitch, const double* init_dev,
                          glt_result* out_dev, void* stream)
{
    if (!t) return invalid("tracker is NULL");
    if (!frame_dev || !init_dev || !out_dev) return invalid("NULL argument");
    if (pitch < t->W[0]) return invalid("pitch < width");
    if (!t->have_points) {
        set_error("glt_set_map_points must come first");
        return GLT_ERR_NO_REFERENCE;
    }
    const int rc = glt_build_pyramid(t, GLT_CUR, frame_dev, pitch, 1, stream);
    if (rc != GLT_OK) return rc;
    // the track kernel is a programmatic dependent of the last pyramid kernel
    // (with one FP32 level the pyramid is a plain copy, and it waits as usual)
    const bool pdl = t->L > 1 || t->packed != nullptr;
    GLT_CHECK(launch_track(t->desc_ptr_dev, t->user_dev, 1, t->cluster, t->threads, track_variant(t->cfg),
                           init_dev, out_dev, reinterpret_cast<cudaStream_t>(stream), pdl),
              "track kernel");
    return GLT_OK;
}

int glt_track_image(glt_tracker* t, const uint8_t* img, int pitch, int is_device, const double T_init[12],
                    const double ab_init[2], glt_result* out, void* stream)
{
    if (!t) return invalid("tracker is NULL");
    if (!img || !out) return invalid("NULL argument");
    if (pitch < t->W[0]) return invalid("pitch < width");
    if (!t->have_points) {
        set_error("glt_set_map_points must come first");
        return GLT_ERR_NO_REFERENCE;
    }
    double Tp[12], abp[2];
    if (!T_init || !ab_init) {
        const int rc = glt_state_predict(&t->state, Tp, abp);
        if (rc != GLT_OK) return rc;
        if (!T_init) T_init = Tp;
        if (!ab_init) ab_init = abp;
    }
    if (!finite_all(T_init, 12) || !finite_all(ab_init, 2)) return invalid("non-finite initial state");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::memcpy(t->h_init, T_init, 12 * sizeof(double));
    t->h_init[12] = ab_init[0];
    t->h_init[13] = ab_init[1];
    GLT_CHECK(cudaMemcpyAsync(t->init_dev, t->h_init, 14 * sizeof(double), cudaMemcpyHostToDevice, s),
              "init upload");
    if (!is_device) {
        const size_t W = (size_t)t->W[0], H = (size_t)t->H[0];
        if ((size_t)pitch == W)
            GLT_CHECK(cudaMemcpyAsync(t->stage_dev, img, W * H, cudaMemcpyHostToDevice, s), "frame upload");
        else
            GLT_CHECK(cudaMemcpy2DAsync(t->stage_dev, W, img, (size_t)pitch, W, H, cudaMemcpyHostToDevice, s),
                      "frame upload");
        img = t->stage_dev;
        pitch = (int)W;
    }
    int rc = glt_track_image_async(t, img, pitch, t->init_dev, t->result_dev, stream);
    if (rc != GLT_OK) return rc;
    GLT_CHECK(cudaMemcpyAsync(t->h_result, t->result_dev, sizeof(glt_result), cudaMemcpyDeviceToHost, s),
              "result download");
    GLT_CHECK(cudaStreamSynchronize(s), "track");
    *out = *t->h_result;
    glt_state_update(&t->state, out);   // a non-finite result leaves the state as it was
    return GLT_OK;
}

int glt_track_frame(glt_tracker* t, const double T_init[12], const double ab_init[2], glt_result* out,
                    void* stream)
{
    int rc = track_prereq(t);
    if (rc != GLT_OK) return rc;
    if (!out) return invalid("NULL argument");
    double Tp[12], abp[2];
    if (!T_init || !ab_init) {
        rc = glt_state_predict(&t->state, Tp, abp);
        if (rc != GLT_OK) return rc;
        if (!T_init) T_init = Tp;
        if (!ab_init) ab_init = abp;
    }
    if (!finite_all(T_init, 12) || !finite_all(ab_init, 2)) return invalid("non-finite initial state");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::memcpy(t->h_init, T_init, 12 * sizeof(double));
    t->h_init[12] = ab_init[0];
    t->h_init[13] = ab_init[1];
    GLT_CHECK(cudaMemcpyAsync(t->init_dev, t->h_init, 14 * sizeof(double), cudaMemcpyHostToDevice, s),
              "init upload");
    GLT_CHECK(launch_track(t->desc_ptr_dev, t->user_dev, 1, t->cluster, t->threads,
                           track_variant(t->cfg), t->init_dev, t->result_dev, s),
              "track kernel");
    GLT_CHECK(cudaMemcpyAsync(t->h_result, t->result_dev, sizeof(glt_result), cudaMemcpyDeviceToHost, s),
              "result download");
    GLT_CHECK(cudaStreamSynchronize(s), "track");
    *out = *t->h_result;
    glt_state_update(&t->state, out);   // a non-finite result leaves the state as it was
    return GLT_OK;
}

// ---------------------------------------------------------------------------
// Tracking state (host only)

static void compose34(const double A[12], const double B[12], double C[12])
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double v = c == 3 ? A[4 * r + 3] : 0.0;
            for (int k = 0; k < 3; ++k) v += A[4 * r + k] * B[4 * k + c];
            C[4 * r + c] = v;
        }
    }
}

// rigid inverse [R^T | -R^T t]
static void inverse34(const double T[12], double Ti[12])
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) Ti[4 * r + c] = T[4 * c + r];
        Ti[4 * r + 3] = -(T[r] * T[3] + T[4 + r] * T[7] + T[8 + r] * T[11]);
    }
}

static bool orthonormalise_rows(double T[12])
{
    double* r0 = T;
    double* r1 = T + 4;
    double* r2 = T + 8;
    const double n0 = std::sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    if (!(n0 > 0.0)) return false;
    for (int i = 0; i < 3; ++i) r0[i] /= n0;
    const double d = r1[0] * r0[0] + r1[1] * r0[1] + r1[2] * r0[2];
    for (int i = 0; i < 3; ++i) r1[i] -= d * r0[i];
    const double n1 = std::sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    if (!(n1 > 0.0)) return false;
    for (int i = 0; i < 3; ++i) r1[i] /= n1;
    r2[0] = r0[1] * r1[2] - r0[2] * r1[1];
    r2[1] = r0[2] * r1[0] - r0[0] * r1[2];
    r2[2] = r0[0] * r1[1] - r0[1] * r1[0];
    return true;
}

static bool state_finite(const glt_state& st)
{
    return finite_all(st.T_cr, 12) && finite_all(st.motion, 12) && std::isfinite(st.a) &&
           std::isfinite(st.b);
}

int glt_state_predict(const glt_state* st, double T_init[12], double ab_init[2])
{
    if (!st || !T_init || !ab_init) return invalid("NULL argument");
    if (!state_finite(*st)) return invalid("non-finite state");
    double T[12];
    compose34(st->motion, st->T_cr, T);
    if (!orthonormalise_rows(T)) return invalid("degenerate rotation in the state");
    std::memcpy(T_init, T, sizeof(T));
    ab_init[0] = st->a;
    ab_init[1] = st->b;
    return GLT_OK;
}

int glt_state_update(glt_state* st, const glt_result* r)
{
    if (!st || !r) return invalid("NULL argument");
    if (!finite_all(r->T, 12) || !std::isfinite(r->a) || !std::isfinite(r->b))
        return invalid("non-finite result");
    double Ti[12];
    inverse34(st->T_cr, Ti);
    compose34(r->T, Ti, st->motion);
    std::memcpy(st->T_cr, r->T, sizeof(st->T_cr));
    st->a = r->a;
    st->b = r->b;
    st->frames += 1;
    return GLT_OK;
}

int glt_get_state(const glt_tracker* t, glt_state* out)
{
    if (!t || !out) return invalid("NULL argument");
    *out = t->state;
    return GLT_OK;
}

int glt_set_state(glt_tracker* t, const glt_state* in)
{
    if (!t || !in) return invalid("NULL argument");
    if (!state_finite(*in) || in->frames < 0) return invalid("non-finite state or frames < 0");
    t->state = *in;
    t->state.reference = t->version;
    return GLT_OK;
}

int glt_debug_linearize(glt_tracker* t, int level, const double T[12], double a, double b,
                        double H[64], double g[8], double* E, int* n, float* res, void* stream)
{
    int rc = track_prereq(t);
    if (rc != GLT_OK) return rc;
    if (level < 0 || level >= t->L) return invalid("level out of range");
    if (!T || !H || !g || !E || !n) return invalid("NULL argument");
    if (!finite_all(T, 12) || !std::isfinite(a) || !std::isfinite(b)) return invalid("non-finite state");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t->N == 0) {
        std::memset(H, 0, 64 * sizeof(double));
        std::memset(g, 0, 8 * sizeof(double));
        *E = 0.0;
        *n = 0;
        return GLT_OK;
    }
    PassParams P;
    make_pass_params(T, a, b, level, P);
    GLT_CHECK(launch_linearize(t, P, res != nullptr, s), "linearize kernel");
    GLT_CHECK(cudaMemcpyAsync(t->h_lin, t->lin_out, kAccPad * sizeof(double), cudaMemcpyDeviceToHost, s),
              "linearize download");
    if (res)
        GLT_CHECK(cudaMemcpyAsync(res, t->lin_res, (size_t)t->N * t->K * sizeof(float), cudaMemcpyDeviceToHost, s),
                  "residual download");
    if (t->Hc) {
        // the cached-Hessian form: H of the level from the reference, the pass's g0 (no e^a)
        double Hl[36];
        GLT_CHECK(cudaMemcpyAsync(Hl, t->Hc + 72 * level, sizeof(Hl), cudaMemcpyDeviceToHost, s),
                  "reference Hessian download");
        GLT_CHECK(cudaStreamSynchronize(s), "linearize");
        const double ea = std::exp(a);
        std::memset(H, 0, 64 * sizeof(double));
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) H[8 * i + j] = ea * ea * Hl[6 * i + j];
        for (int i = 0; i < 8; ++i) g[i] = i < 6 ? ea * t->h_lin[i] : 0.0;
        *E = t->h_lin[kHcE];
        *n = (int)t->h_lin[kHcN];
        return GLT_OK;
    }
    GLT_CHECK(cudaStreamSynchronize(s), "linearize");
    int idx = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = i; j < 8; ++j) {
            H[8 * i + j] = t->h_lin[idx];
            H[8 * j + i] = t->h_lin[idx];
            ++idx;
        }
    for (int i = 0; i < 8; ++i) g[i] = t->h_lin[kIdxG + i];
    *E = t->h_lin[kIdxE];
    *n = (int)t->h_lin[kIdxN];
    return GLT_OK;
}

int glt_get_shape(const glt_tracker* t, int* cluster, int* threads)
{
    if (!t || !cluster || !threads) return invalid("NULL argument");
    *cluster = t->cluster;
    *threads = t->threads;
    return GLT_OK;
}

int glt_get_pyramid(glt_tracker* t, int slot, int level, uint8_t* out, void* stream)
{
    if (!t || !out) return invalid("NULL argument");
    if (slot != GLT_REF && slot != GLT_CUR) return invalid("bad slot");
    if (level < 0 || level >= t->L) return invalid("level out of range");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Pyramid& P = t->pyr[slot];
    GLT_CHECK(cudaMemcpy2DAsync(out, (size_t)t->W[level], P.base + P.off[level], (size_t)t->pitch[level],
                                (size_t)t->W[level], (size_t)t->H[level], cudaMemcpyDeviceToHost, s),
              "pyramid download");
    GLT_CHECK(cudaStreamSynchronize(s), "pyramid download");
    return GLT_OK;
}

int glt_get_trace(glt_tracker* t, double* cost, int* info, int max, int* count, void* stream)
{
    if (!t || !count || max < 0 || (max > 0 && (!cost || !info))) return invalid("bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int passes = 0;
    GLT_CHECK(cudaMemcpyAsync(&passes, t->trace_count, sizeof(int), cudaMemcpyDeviceToHost, s), "trace");
    GLT_CHECK(cudaStreamSynchronize(s), "trace");
    int k = std::min(std::min(passes, t->max_trace), max);
    if (k > 0) {
        std::vector<int> nn(k);
        GLT_CHECK(cudaMemcpyAsync(cost, t->trace_E, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s), "trace");
        GLT_CHECK(cudaMemcpyAsync(nn.data(), t->trace_n, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, s), "trace");
        GLT_CHECK(cudaMemcpyAsync(info, t->trace_info, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, s), "trace");
        GLT_CHECK(cudaStreamSynchronize(s), "trace");
        for (int i = 0; i < k; ++i)
            cost[i] = (nn[i] >= t->cfg.min_valid && nn[i] > 0) ? cost[i] / nn[i] : INFINITY;
    }
    *count = k;
    return GLT_OK;
}

// ---------------------------------------------------------------------------
// batched form
// ---------------------------------------------------------------------------
static void free_batch(glt_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (int k = 0; k < kMaxBatchClasses - 1; ++k) {
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
        if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
    }
    cudaFree(b->descs_dev);
    cudaFree(b->users_dev);
    cudaFree(b->copy_dev);
    cudaFree(b->jobs_dev);
    cudaFree(b->tile_map_dev);
    cudaFree(b->pack_dev);
    cudaFree(b->prop_jobs);
    cudaFree(b->prop_init);
    delete b;
}

int glt_batch_create(glt_tracker* const* trackers, int S, glt_batch** out)
{
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    if (!trackers || S < 1 || S > 65535) return invalid("need 1..65535 trackers");
    const int prec = trackers[0] ? trackers[0]->cfg.precision : -1;
    for (int i = 0; i < S; ++i) {
        if (!trackers[i]) return invalid("NULL tracker in batch");
        if (trackers[i]->cfg.precision != prec) return invalid("all trackers of a batch need the same precision");
        if (trackers[i]->device != trackers[0]->device) return invalid("all trackers must be on one device");
        if ((trackers[i]->Hc != nullptr) != (trackers[0]->Hc != nullptr))
            return invalid("all or none of the trackers of a batch need GLT_HESSIAN_CACHED");
    }
    glt_batch* b = new glt_batch();
    b->S = S;
    b->precision = prec;
    b->trk.assign(trackers, trackers + S);
    b->order.resize(S);
    for (int i = 0; i < S; ++i) b->order[i] = i;
    // heaviest streams first: a pass costs about its residual samples (point
    // capacity x samples per point); the frame size breaks ties
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const double wx = (double)trackers[x]->cfg.max_points * trackers[x]->K;
        const double wy = (double)trackers[y]->cfg.max_points * trackers[y]->K;
        if (wx != wy) return wx > wy;
        return trackers[x]->cfg.width > trackers[y]->cfg.width;
    });
    for (int i = 0; i < S; ++i) b->Lmax = std::max(b->Lmax, trackers[i]->L);
#define BALLOC(call)                                  \
    do {                                              \
        cudaError_t e2 = (call);                      \
        if (e2 != cudaSuccess) {                      \
            free_batch(b);                            \
            return cuda_fail(e2, "batch allocation"); \
        }                                             \
    } while (0)
    std::vector<StreamDesc*> dp(S);
    std::vector<int> users(S);
    for (int i = 0; i < S; ++i) {
        dp[i] = trackers[b->order[i]]->desc_dev;
        users[i] = b->order[i];
    }
    BALLOC(dalloc(&b->descs_dev, (size_t)S));
    BALLOC(dalloc(&b->users_dev, (size_t)S));
    BALLOC(cudaMemcpy(b->descs_dev, dp.data(), S * sizeof(StreamDesc*), cudaMemcpyHostToDevice));
    BALLOC(cudaMemcpy(b->users_dev, users.data(), S * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<CopyJob> copies(S);
    std::vector<PyrJob> jobs((size_t)std::max(1, b->Lmax - 1) * S);
    std::vector<PackJob> packs((size_t)b->Lmax * S);
    for (int i = 0; i < S; ++i) {
        glt_tracker* t = trackers[i];
        copies[i].dst = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[0];
        copies[i].W = t->W[0];
        copies[i].H = t->H[0];
        copies[i].dp = t->pitch[0];
        for (int l = 1; l < b->Lmax; ++l) {
            PyrJob& J = jobs[(size_t)(l - 1) * S + i];
            std::memset(&J, 0, sizeof(J));
            if (l < t->L) {
                J.src = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l - 1];
                J.dst = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l];
                J.sW = t->W[l - 1];
                J.sH = t->H[l - 1];
                J.sp = t->pitch[l - 1];
                J.dW = t->W[l];
                J.dH = t->H[l];
                J.dp = t->pitch[l];
            }
        }
        for (int l = 0; l < b->Lmax; ++l) {
            PackJob& P = packs[(size_t)l * S + i];
            std::memset(&P, 0, sizeof(P));
            if (l < t->L && t->packed) {
                P.src = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l];
                P.dst = t->packed + t->poff[l];
                P.W = t->W[l];
                P.H = t->H[l];
                P.sp = t->pitch[l];
            }
        }
    }
    // per round, every output tile of every stream as (stream << 16) | tile:
    // one CTA per entry in the batched pyramid kernel
    const int rounds = std::max(1, b->Lmax - 1);
    std::vector<unsigned> tmap;
    for (int r = 0; r < rounds; ++r) {
        b->tile_map_off[r] = tmap.size();
        for (int i = 0; i < S; ++i) {
            const PyrJob& J = jobs[(size_t)r * S + i];
            const int n = pyr_tiles_x(J.dW) * pyr_tiles_y(J.dH);
            for (int k = 0; k < n; ++k) tmap.push_back(((unsigned)i << 16) | (unsigned)k);
        }
        b->tile_total[r] = (int)(tmap.size() - b->tile_map_off[r]);
    }
    if (tmap.empty()) tmap.push_back(0u);
    BALLOC(dalloc(&b->tile_map_dev, tmap.size()));
    BALLOC(cudaMemcpy(b->tile_map_dev, tmap.data(), tmap.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    BALLOC(dalloc(&b->copy_dev, (size_t)S));
    BALLOC(dalloc(&b->jobs_dev, jobs.size()));
    BALLOC(dalloc(&b->pack_dev, packs.size()));
    BALLOC(cudaMemcpy(b->copy_dev, copies.data(), S * sizeof(CopyJob), cudaMemcpyHostToDevice));
    BALLOC(cudaMemcpy(b->jobs_dev, jobs.data(), jobs.size() * sizeof(PyrJob), cudaMemcpyHostToDevice));
    BALLOC(cudaMemcpy(b->pack_dev, packs.data(), packs.size() * sizeof(PackJob), cudaMemcpyHostToDevice));
#undef BALLOC
    // one kernel variant for the whole batch: the most general one any stream needs
    b->variant = 0;
    for (int i = 0; i < S; ++i) {
        const int v = track_variant(trackers[i]->cfg);
        if (v == 1 || v == 2 || v == 4) b->variant = v;
        else if (v == 3 && b->variant == 0) b->variant = 3;
    }
    {
        int cl = 2, th = b->variant == 4 ? 512 : 256;   // the cached-Hessian kernel's only width
        if (!track_shape_ok(cl, th, b->variant)) cl = 1;
        set_uniform(b, cl, th);
    }
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int k = 0; k < kMaxBatchClasses - 1 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch stream / events");
    }
    *out = b;
    return GLT_OK;
}

// The track launch(es) of a batch: one launch when there is one class, else
// class 0 on `s` and class k > 0 on side stream aux[k - 1], each forked from
// and joined back into `s` (under stream capture: parallel graph nodes).
// pdl applies to the launch on `s` (the single launch, or class 0: the
// heaviest streams, whose setup then overlaps the pyramids); the side
// classes wait for the fork point to complete.
static cudaError_t launch_batch_track(glt_batch* b, const double* init, glt_result* out,
                                      cudaStream_t s, bool pdl)
{
    if (b->nclass == 1)
        return launch_track(b->descs_dev, b->users_dev, b->S, b->cls_cluster[0], b->cls_threads[0],
                            b->variant, init, out, s, pdl);
    cudaError_t e = cudaEventRecord(b->ev_fork, s);
    for (int k = 1; k < b->nclass && e == cudaSuccess; ++k) {
        const int f = b->cls_first[k], n = b->cls_first[k + 1] - f;
        e = cudaStreamWaitEvent(b->aux[k - 1], b->ev_fork, 0);
        if (e == cudaSuccess)
            e = launch_track(b->descs_dev + f, b->users_dev + f, n, b->cls_cluster[k], b->cls_threads[k],
                             b->variant, init, out, b->aux[k - 1], false);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[k - 1], b->aux[k - 1]);
    }
    if (e == cudaSuccess)
        e = launch_track(b->descs_dev, b->users_dev, b->cls_first[1], b->cls_cluster[0], b->cls_threads[0],
                         b->variant, init, out, s, pdl);
    for (int k = 1; k < b->nclass && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s, b->ev_join[k - 1], 0);
    return e;
}

static void drop_graph(glt_batch* b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
}

void glt_batch_destroy(glt_batch* b) { free_batch(b); }

static int batch_pyramid(glt_batch* b, const uint8_t* const* frames_dev, cudaStream_t s)
{
    int maxbytes = 0, maxpix = 0;
    for (glt_tracker* t : b->trk) {
        maxbytes = std::max(maxbytes, t->W[0] * t->H[0]);
        maxpix = std::max(maxpix, t->W[0] * t->H[0]);
    }
    // level 1 reads the frames and writes level 0; streams with one level
    // only need the copy
    bool single_level = false;
    for (glt_tracker* t : b->trk) single_level |= t->L == 1;
    // every launch after the first is a programmatic dependent of the previous one
    bool after_first = false;
    if (single_level || b->Lmax == 1) {
        GLT_CHECK(launch_copy_frames(frames_dev, b->copy_dev, b->S, maxbytes, s), "batch copy kernel");
        after_first = true;
    }
    for (int l = 1; l < b->Lmax; ++l) {
        GLT_CHECK(launch_pyr_down(b->jobs_dev + (size_t)(l - 1) * b->S,
                                  b->tile_map_dev + b->tile_map_off[l - 1], b->tile_total[l - 1],
                                  s, (l == 1 && !single_level) ? frames_dev : nullptr,
                                  nullptr, 0, after_first),
                  "batch pyramid kernel");
        after_first = true;
    }
    if (b->precision == GLT_MIXED)
        GLT_CHECK(launch_pack(b->pack_dev, b->Lmax * b->S, maxpix, s, after_first), "batch pack kernel");
    for (glt_tracker* t : b->trk) t->pyr[GLT_CUR].built = true;
    return GLT_OK;
}

int glt_batch_build_pyramid(glt_batch* b, const uint8_t* const* frames_dev, void* stream)
{
    if (!b || !frames_dev) return invalid("NULL argument");
    return batch_pyramid(b, frames_dev, reinterpret_cast<cudaStream_t>(stream));
}

static int batch_prereq(glt_batch* b)
{
    if (!b) return invalid("batch is NULL");
    for (glt_tracker* t : b->trk)
        if (!t->have_points) {
            set_error("every tracker of the batch needs map points");
            return GLT_ERR_NO_REFERENCE;
        }
    return GLT_OK;
}

int glt_batch_track(glt_batch* b, const double* init_dev, glt_result* out_dev, void* stream)
{
    int rc = batch_prereq(b);
    if (rc != GLT_OK) return rc;
    if (!init_dev || !out_dev) return invalid("NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (b->nn) {
        GLT_CHECK(launch_proposal(b, init_dev, s), "proposal kernels");
        init_dev = b->prop_init;
    }
    GLT_CHECK(launch_batch_track(b, init_dev, out_dev, s, false), "batch track kernel");
    return GLT_OK;
}

int glt_batch_capture(glt_batch* b, const uint8_t* const* frames_dev, const double* init_dev,
                      glt_result* out_dev, void* stream)
{
    int rc = batch_prereq(b);
    if (rc != GLT_OK) return rc;
    if (!frames_dev || !init_dev || !out_dev) return invalid("NULL argument");
    if (!stream) return invalid("graph capture needs a non-default stream");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    GLT_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    int r1 = batch_pyramid(b, frames_dev, s);
    cudaError_t e1 = cudaSuccess;
    if (b->nn) {
        e1 = launch_proposal(b, init_dev, s);
        init_dev = b->prop_init;
    }
    // without the proposal stage the track kernel follows the last pyramid
    // kernel as its programmatic dependent (its setup overlaps the pyramids);
    // after the proposal stage it reads that stage's output from its first
    // instruction, so it waits as usual
    if (e1 == cudaSuccess) e1 = launch_batch_track(b, init_dev, out_dev, s, b->nn == nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (r1 != GLT_OK) {
        if (g) cudaGraphDestroy(g);
        return r1;
    }
    if (e1 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e1, "capture track kernel");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    b->graph = g;
    GLT_CHECK(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    return GLT_OK;
}

int glt_batch_replay(glt_batch* b, void* stream)
{
    if (!b || !b->exec) return invalid("no captured graph");
    GLT_CHECK(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)), "graph launch");
    return GLT_OK;
}

int glt_batch_set_shape(glt_batch* b, int cluster, int threads)
{
    if (!b) return invalid("batch is NULL");
    if (!track_shape_ok(cluster, threads, b->variant)) return invalid("shape cannot launch");
    set_uniform(b, cluster, threads);
    drop_graph(b);
    return GLT_OK;
}

int glt_batch_set_classes(glt_batch* b, int heavy, int heavy_cluster, int heavy_threads,
                          int light_cluster, int light_threads)
{
    if (!b) return invalid("batch is NULL");
    if (heavy < 0 || heavy > b->S) return invalid("heavy must be in [0, S]");
    if ((heavy > 0 && !track_shape_ok(heavy_cluster, heavy_threads, b->variant)) ||
        (heavy < b->S && !track_shape_ok(light_cluster, light_threads, b->variant)))
        return invalid("shape cannot launch");
    apply_table(b, split_table(b->S, heavy, heavy_cluster, heavy_threads, light_cluster, light_threads));
    drop_graph(b);
    return GLT_OK;
}

int glt_batch_set_proportional(glt_batch* b, int points_per_cta, int threads)
{
    if (!b) return invalid("batch is NULL");
    if (points_per_cta < 1) return invalid("points_per_cta must be >= 1");
    ClassTable c;
    if (!proportional_table(b, points_per_cta, threads, c)) return invalid("threads cannot launch");
    apply_table(b, c);
    drop_graph(b);
    return GLT_OK;
}

int glt_batch_get_classes(const glt_batch* b, int* heavy, int* heavy_cluster, int* heavy_threads,
                          int* light_cluster, int* light_threads)
{
    if (!b) return invalid("batch is NULL");
    const int k1 = b->nclass > 1 ? 1 : 0;
    if (heavy) *heavy = b->nclass > 1 ? b->cls_first[1] : b->S;
    if (heavy_cluster) *heavy_cluster = b->cls_cluster[0];
    if (heavy_threads) *heavy_threads = b->cls_threads[0];
    if (light_cluster) *light_cluster = b->cls_cluster[k1];
    if (light_threads) *light_threads = b->cls_threads[k1];
    return GLT_OK;
}

int glt_batch_get_class_table(const glt_batch* b, int max, int* first, int* cluster, int* threads,
                              int* nclass)
{
    if (!b || !nclass) return invalid("NULL argument");
    if (max < 0) return invalid("max must be >= 0");
    *nclass = b->nclass;
    for (int k = 0; k < b->nclass && k < max; ++k) {
        if (first) first[k] = b->cls_first[k];
        if (cluster) cluster[k] = b->cls_cluster[k];
        if (threads) threads[k] = b->cls_threads[k];
    }
    return GLT_OK;
}

int glt_batch_autotune(glt_batch* b, const double* init_dev, glt_result* out_dev, int reps,
                       int* best_cluster, int* best_threads, float* best_ms, void* stream)
{
    int rc = batch_prereq(b);
    if (rc != GLT_OK) return rc;
    if (!init_dev || !out_dev || reps < 1) return invalid("bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the batch's signature: kernel variant and, in launch order, every
    // stream's frame size, point capacity and level count
    std::string key = std::to_string(b->variant);
    for (int i = 0; i < b->S; ++i) {
        const glt_tracker* t = b->trk[b->order[i]];
        key += "|" + std::to_string(t->W[0]) + "x" + std::to_string(t->H[0]) + "x" +
               std::to_string(t->cfg.max_points) + "x" + std::to_string(t->L);
    }
    TuneResult best{};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        // candidates: one shape for every stream; a heavy class (the first
        // quarter or half of the launch order) with a wide shape and the light
        // rest with a narrow one; clusters in proportion to each stream's
        // points (glt_batch_set_proportional) at several points per CTA
        const int uniform[][2] = {{1, 128}, {1, 256}, {2, 128}, {2, 256}, {4, 128}, {4, 256},
                                  {8, 128}, {8, 256}, {1, 512}, {2, 512}, {4, 512}, {8, 512}};
        const int wide[][2] = {{8, 128}, {16, 128}, {8, 256}, {4, 512}, {8, 512}};
        const int narrow[][2] = {{1, 128}, {2, 128}, {4, 128}, {8, 128}, {2, 256}, {2, 512}};
        const int prop[][2] = {{256, 128}, {320, 128}, {384, 128}, {448, 128}, {512, 128}, {768, 128},
                               {512, 256}, {768, 256}, {1024, 256}, {1024, 512}, {1536, 512}};
        std::vector<TuneResult> cands;
        for (auto& u : uniform)
            if (track_shape_ok(u[0], u[1], b->variant)) cands.push_back(uniform_table(b->S, u[0], u[1]));
        if (b->S >= 4) {
            for (int part = 4; part >= 2; part /= 2) {
                const int heavy = std::max(1, b->S / part);
                for (auto& w : wide) {
                    if (!track_shape_ok(w[0], w[1], b->variant)) continue;
                    for (auto& n : narrow)
                        if (track_shape_ok(n[0], n[1], b->variant))
                            cands.push_back(split_table(b->S, heavy, w[0], w[1], n[0], n[1]));
                }
            }
        }
        if (b->S >= 2) {
            for (auto& pp : prop) {
                ClassTable c;
                if (proportional_table(b, pp[0], pp[1], c) && c.nclass > 1) cands.push_back(c);
            }
        }
        cudaEvent_t e0, e1;
        GLT_CHECK(cudaEventCreate(&e0), "event");
        GLT_CHECK(cudaEventCreate(&e1), "event");
        best.ms = 1e30f;
        for (TuneResult& c : cands) {
            apply_table(b, c);
            cudaError_t e = launch_batch_track(b, init_dev, out_dev, s, false);   // warm-up
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r) launch_batch_track(b, init_dev, out_dev, s, false);
            cudaEventRecord(e1, s);
            cudaError_t es = cudaEventSynchronize(e1);
            if (es != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(es, "autotune");
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            c.ms = ms / reps;
            if (c.ms < best.ms) best = c;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best.ms >= 1e30f) return invalid("no shape could launch");
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    apply_table(b, best);
    drop_graph(b);
    if (best_cluster) *best_cluster = best.cluster[0];
    if (best_threads) *best_threads = best.threads[0];
    if (best_ms) *best_ms = best.ms;
    return GLT_OK;
}

}  // extern "C"

// Host-side internals shared by the library's translation units: the tracker
// and batch objects and the kernel launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "glt.h"
#include "glt_device.cuh"

namespace glt {

// per-slot pyramid storage: one allocation, level l at off[l], row pitch pitch[l]
struct Pyramid {
    uint8_t* base = nullptr;
    size_t bytes = 0;
    size_t off[kMaxLevels] = {};
    bool built = false;
};

struct PyrJob {             // one "level l-1 -> level l" downsampling job
    const uint8_t* src;
    uint8_t* dst;
    int sW, sH, sp;
    int dW, dH, dp;
};

struct CopyJob {            // one frame -> level-0 copy (batched form)
    uint8_t* dst;
    int W, H, dp;
};

struct PropJob {            // coarsest levels (40 x 30) of one stream, for the proposal input
    const uint8_t* ref;
    const uint8_t* cur;
    int pitch;
};

// launch classes of a batch: at most one per cluster size 16, 8, 4, 2, 1
constexpr int kMaxBatchClasses = 5;

struct PackJob {            // one level -> FP16 (I, gx, gy, 0) copy (mixed form)
    const uint8_t* src;
    uint2* dst;
    int W, H, sp;
};

}  // namespace glt

struct glt_tracker {
    glt_config cfg;
    int device = 0;
    int L = 0;
    int W[glt::kMaxLevels] = {}, H[glt::kMaxLevels] = {}, pitch[glt::kMaxLevels] = {};
    glt::Pyramid pyr[2];
    uint2* packed = nullptr;              // CUR FP16 levels (GLT_MIXED)
    size_t poff[glt::kMaxLevels] = {};    // pixel offsets into `packed`
    float* uvd_dev = nullptr;             // staging for host map points
    float4* pt = nullptr;
    float2* dz = nullptr;
    float* I0 = nullptr;
    float2* G0 = nullptr;                 // GLT_IC reference gradients [L][Npad][K]
    double* Hc = nullptr;                 // GLT_HESSIAN_CACHED: per level H, H^-1 [L][72]
    int K = 8;                            // samples per point of the pattern
    int Npad = 0;
    int N = 0;
    bool have_points = false;
    glt::StreamDesc desc_host{};
    glt::StreamDesc* desc_dev = nullptr;
    glt::StreamDesc** desc_ptr_dev = nullptr;  // device array {desc_dev}
    int* user_dev = nullptr;                   // device {0}
    int* trace_count = nullptr;
    unsigned version = 0;                      // bumped by set_map_points
    glt::PyrJob* jobs_dev = nullptr;      // [2 slots][L-1] downsampling jobs
    glt::PackJob* pack_dev = nullptr;     // L packing jobs
    double* init_dev = nullptr;           // 14 doubles
    glt_result* result_dev = nullptr;
    double* trace_E = nullptr;
    int* trace_n = nullptr;
    int* trace_info = nullptr;
    int max_trace = 0;
    // single-pass multi-block linearisation (debug / parity)
    float* lin_partials = nullptr;
    unsigned* lin_counter = nullptr;
    double* lin_out = nullptr;
    float* lin_res = nullptr;
    uint8_t* stage_dev = nullptr;         // device copy of a host frame (glt_build_pyramid)
    int lin_blocks = 0;
    // pinned host staging
    double* h_init = nullptr;
    glt_result* h_result = nullptr;
    double* h_lin = nullptr;
    int cluster = 1, threads = 256;
    glt_state state{};                    // host-side tracking state (glt_get_state)
};

struct glt_batch {
    std::vector<glt_tracker*> trk;        // caller order
    std::vector<int> order;               // launch order (descending work)
    int S = 0;
    int precision = GLT_FP32;
    glt::StreamDesc** descs_dev = nullptr; // launch order: each tracker's device descriptor
    int* users_dev = nullptr;              // launch order -> caller index
    glt::CopyJob* copy_dev = nullptr;     // caller order
    glt::PyrJob* jobs_dev = nullptr;      // [L-1 rounds][S] caller order
    unsigned* tile_map_dev = nullptr;     // per round: (stream << 16) | tile, for every tile
    size_t tile_map_off[GLT_MAX_LEVELS] = {};  // offset of round l-1 in tile_map_dev
    int tile_total[GLT_MAX_LEVELS] = {};  // tiles of round l-1 over all streams
    glt::PackJob* pack_dev = nullptr;     // [Lmax][S]
    int Lmax = 0;
    int variant = 0;                      // kernel variant (track_variant of the streams)
    // launch classes over the launch order: class k = the streams
    // [cls_first[k], cls_first[k + 1]), each class with its own (cluster,
    // threads); the classes run as concurrent launches (graph branches):
    // class 0 on the caller's stream, class k > 0 on side stream aux[k - 1]
    int nclass = 1;
    int cls_first[glt::kMaxBatchClasses + 1] = {};
    int cls_cluster[glt::kMaxBatchClasses] = {};
    int cls_threads[glt::kMaxBatchClasses] = {};
    cudaStream_t aux[glt::kMaxBatchClasses - 1] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[glt::kMaxBatchClasses - 1] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // learned initial-pose proposal (optional)
    glt_nn* nn = nullptr;
    const double* motion_dev = nullptr;   // [S][12] each stream's last inter-frame motion
    glt::PropJob* prop_jobs = nullptr;
    double* prop_init = nullptr;
};

namespace glt {

void set_error(const std::string& msg);
int invalid_arg_msg(const char* msg);
cudaError_t nn_forward(glt_nn* n, const float* x, const float* mo, int B, cudaStream_t s);
cudaError_t launch_proposal(glt_batch* b, const double* init_dev, cudaStream_t s);
int cuda_fail(cudaError_t e, const char* what);

// pyramid.cu
// pyramid-family launches; pdl as for launch_track (the kernels wait for
// their predecessor before reading what it writes)
// launch_pyr_down: one level, `total` output tiles over all jobs;
// tile_map_dev[f] = (job << 16) | tile within the job, or NULL for one job
cudaError_t launch_pyr_down(const PyrJob* jobs_dev, const unsigned* tile_map_dev, int total,
                            cudaStream_t s, const uint8_t* const* frames = nullptr,
                            const uint8_t* src = nullptr, int sp = 0, bool pdl = false);
cudaError_t launch_copy_frames(const uint8_t* const* frames, const CopyJob* jobs, int njobs,
                               int max_bytes, cudaStream_t s, bool pdl = false);
cudaError_t launch_pack(const PackJob* jobs, int njobs, int max_pixels, cudaStream_t s,
                        bool pdl = false);
__host__ __device__ int pyr_tiles_x(int dW);
__host__ __device__ int pyr_tiles_y(int dH);

// points.cu
cudaError_t launch_set_points(const glt_tracker* t, const float* uvd_dev, int n, cudaStream_t s);
// per-reference Hessian of every level and its inverse (GLT_HESSIAN_CACHED)
cudaError_t launch_ic_hessian(const glt_tracker* t, cudaStream_t s);

#ifdef GLT_CHECKED
// bounds-checked build: each translation unit's check flags (CheckSite bits),
// read and cleared
unsigned check_flags_track();
unsigned check_flags_pyramid();
unsigned check_flags_points();
#endif

// track.cu
// kernel variant of a configuration: 0 FP32 forward, 1 GLT_MIXED, 2 FP32 with
// p x p patches, 3 FP32 inverse compositional, 4 the cached Hessian (FP32, IC)
inline int track_variant(const glt_config& c)
{
    return c.hessian == GLT_HESSIAN_CACHED ? 4
         : c.precision == GLT_MIXED ? 1 : c.pattern != 0 ? 2 : c.jacobian == GLT_IC ? 3 : 0;
}
// pdl: launch as a programmatic dependent of the previous kernel in the
// stream (cudaLaunchAttributeProgrammaticStreamSerialization): the kernel may
// start while that kernel runs and waits for its results on the device
// (griddepcontrol.wait) before it reads them.  Only for launches whose
// predecessor is one of the library's pyramid kernels.
cudaError_t launch_track(const StreamDesc* const* descs, const int* users, int S, int cluster,
                         int threads, int variant, const double* init, glt_result* results,
                         cudaStream_t s, bool pdl = false);
cudaError_t launch_linearize(const glt_tracker* t, const PassParams& P, bool want_res,
                             cudaStream_t s);
bool track_shape_ok(int cluster, int threads, int variant);
// the fixed part of `passes` tracker passes (no points) in solve mode
// `solve`, CTA 0's cycles to *cycles (-1 when an exchange wait ran out);
// drop_rank >= 0: that CTA withholds its first partial, so every wait of the
// cluster runs out
cudaError_t launch_pass_floor(int cluster, int threads, bool cached, int passes, long long* cycles,
                              cudaStream_t s, int drop_rank = -1, int solve = GLT_SOLVE_FP64);

}  // namespace glt

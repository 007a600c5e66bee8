// tune.cu -- autotuner of the mixed path's far field.
//
// The paper runs its FMM at one fixed precision (Sec. 4.4).  Here the far
// field of the mixed path is either the direct tiled sum or the treecode,
// and the treecode's speed and error depend on its Chebyshev degree and
// opening parameter in a way that varies with the mesh (grading, curvature,
// size) and with the density of the targets.  The tuner measures instead of
// modelling: on a sample of the caller's targets it times every candidate
// with CUDA events and compares its Phi with the float-float path (the
// direct sum to FP64 accuracy), then keeps the fastest candidate within the
// error budget.  The sample is a few windows of consecutive Morton-sorted
// targets, so its blocks of targets are as compact as in the full workload
// and a candidate's interaction lists (and cost per target) are the ones it
// would have there.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kTuneWindow = 4096;   // targets per window (16 blocks of the mixed kernel)
constexpr int kTuneWindows = 8;

struct Candidate {
    int mode;      // 0 direct, 1 treecode
    int degree;
    float theta;
};
const Candidate kCandidates[] = {
    {0, 0, 0.0f},    {1, 5, 0.35f},  {1, 6, 0.4f},  {1, 6, 0.45f},  {1, 7, 0.4f},
    {1, 7, 0.45f},   {1, 7, 0.5f},   {1, 8, 0.45f}, {1, 8, 0.5f},   {1, 10, 0.55f},
};

// max |a - b| over n entries, as the bit pattern of a non-negative double
// (ordered like the values)
__global__ void k_max_abs_diff(const double* __restrict__ a, const double* __restrict__ b, int n,
                               unsigned long long* __restrict__ out)
{
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = fabs(a[i] - b[i]);
        m = d > m || d != d ? d : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m || v != v ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int max_abs_diff(Ctx* ctx, const double* a, const double* b, int n, unsigned long long* d_word, double* out,
                 cudaStream_t st)
{
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(d_word, 0, sizeof(unsigned long long), st));
    k_max_abs_diff<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(a, b, n, d_word);
    LSM_LAUNCHED(ctx);
    unsigned long long w = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&w, d_word, sizeof(w), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    double v;
    std::memcpy(&v, &w, sizeof(v));
    *out = v;
    return LSM_OK;
}

}  // namespace

int autotune_sorted(Ctx* ctx, Mesh* me, const Targets& t, double budget, lsm_tune_result* res, cudaStream_t st)
{
    // the sample: windows of consecutive sorted targets, evenly spread
    const int win = std::min(kTuneWindow, t.n);
    const int nw = std::max(1, std::min(kTuneWindows, t.n / std::max(1, win)));
    const int m = nw * win;
    Scratch s(st);
    double *S = nullptr, *Rref = nullptr, *R = nullptr;
    unsigned long long* word = nullptr;
    LSM_CUDA_TRY(ctx, s.get(&S, 3 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&Rref, 4 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&word, 1));
    for (int w = 0; w < nw; w++) {
        const int64_t off = nw > 1 ? (int64_t)(t.n - win) * w / (nw - 1) : 0;
        for (int c = 0; c < 3; c++)
            LSM_CUDA_TRY(ctx, cudaMemcpyAsync(S + (size_t)c * m + (size_t)w * win, t.x + c * t.ld + off,
                                              sizeof(double) * win, cudaMemcpyDeviceToDevice, st));
    }
    Targets ts{S, m, m};
    int rc = eval_sorted(ctx, me, ts, Rref, LSM_FF, st);
    if (rc != LSM_OK) return rc;

    cudaEvent_t e0, e1;
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e0));
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e1));
    struct Meas {
        Candidate c;
        double ms, err;
    };
    std::vector<Meas> meas;
    const int saved_mode = me->tune_mode, saved_deg = me->tune_degree;
    const float saved_theta = me->tune_theta;
    for (const Candidate& c : kCandidates) {
        me->tune_mode = c.mode;
        me->tune_degree = c.degree;
        me->tune_theta = c.theta;
        // the first evaluation builds the candidate's tree; the second is timed
        rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);
        if (rc == LSM_OK) {
            cudaEventRecord(e0, st);
            rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);
            cudaEventRecord(e1, st);
        }
        if (rc != LSM_OK) break;
        double err = 0.0;
        rc = max_abs_diff(ctx, R, Rref, m, word, &err, st);
        if (rc != LSM_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        meas.push_back(Meas{c, (double)ms, err});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LSM_OK) {
        me->tune_mode = saved_mode;
        me->tune_degree = saved_deg;
        me->tune_theta = saved_theta;
        return rc;
    }
    // fastest within the budget; else the most accurate
    int best = -1;
    for (int i = 0; i < (int)meas.size(); i++)
        if (meas[i].err <= budget && (best < 0 || meas[i].ms < meas[best].ms)) best = i;
    if (best < 0) {
        best = 0;
        for (int i = 1; i < (int)meas.size(); i++)
            if (meas[i].err < meas[best].err) best = i;
    }
    const Candidate& c = meas[best].c;
    me->tune_mode = c.mode;
    me->tune_degree = c.degree;
    me->tune_theta = c.theta;
    if (c.mode == 1) {
        rc = tree_ensure(ctx, me, st, false);
        if (rc != LSM_OK) return rc;
    }
    if (res) {
        res->use_tree = c.mode;
        res->tree_degree = c.degree;
        res->tree_theta = c.theta;
        res->candidates = (int32_t)meas.size();
        res->sample_targets = m;
        res->err_phi = meas[best].err;
        res->ms_sample = meas[best].ms;
        res->ms_direct = meas[0].ms;
        res->err_direct = meas[0].err;
    }
    return LSM_OK;
}

}  // namespace lsm

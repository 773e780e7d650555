// rs_check.cu -- device-side checks: the RS_CHECK table check that runs
// before every resample of a plan created with RS_CHECK, and the bounded-wait
// self-test.
//
// The table check verifies, per output of both axes, what every pass kernel
// relies on when it reads a window: the window lies in the input
// (0 <= start <= n_in - t_eff), its working-precision weights are finite and
// sum to one (within 1e-5 for FP32 working precision, 1e-12 for FP64).  A
// failing output sets the plan's error word to kErrCheck, which rs_plan_check
// reports as RS_ERR_DEVICE; the resample itself still runs.
//
// The wait self-test runs the bounded mbarrier wait that every kernel uses on
// a barrier nobody arrives on, with a short limit: it must give up, set the
// plan's error word to the timeout code and return, leaving the context
// usable.
#include "rs_plan.h"

namespace rs {
namespace {

template <typename W>
__global__ void table_check_kernel(AxisGeom g, const int32_t *start, const W *w, double tol, int *err)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= g.n_out) return;
    const int64_t s = start[i];
    bool ok = s >= 0 && s <= g.n_in - g.t_eff;
    double sum = 0.0;
    for (int k = 0; k < g.t_eff; ++k) {
        const double v = double(w[i * g.t_eff + k]);
        ok = ok && isfinite(v);
        sum += v;
    }
    ok = ok && fabs(sum - 1.0) <= tol;
    if (!ok) fused::flag(err, fused::kErrCheck);
}

__global__ void wait_selftest_kernel(uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        fused::mbar_init(&bar, 1); // one arrival expected; none comes
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    fused::wait_or_abort(&bar, 0, &abort_flag, err, limit_ns);
}

} // namespace

cudaError_t launch_table_check(const rs_plan *p, cudaStream_t s)
{
    for (int axis = 0; axis < 2; ++axis) {
        const AxisGeom &g = axis == 0 ? p->gy : p->gx;
        const AxisTables &t = axis == 0 ? p->ty : p->tx;
        const unsigned blocks = unsigned((g.n_out + 255) / 256);
        if (p->work_double)
            table_check_kernel<double><<<blocks, 256, 0, s>>>(g, t.start, static_cast<const double *>(t.wwork),
                                                              1e-12, p->d_err);
        else
            table_check_kernel<float><<<blocks, 256, 0, s>>>(g, t.start, static_cast<const float *>(t.wwork), 1e-5,
                                                             p->d_err);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_wait_selftest(int *err, uint64_t limit_ns, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(limit_ns, err);
    return cudaGetLastError();
}

} // namespace rs

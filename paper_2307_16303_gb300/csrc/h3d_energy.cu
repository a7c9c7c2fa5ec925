// h3d_energy.cu -- energy of charges under the compressed operator and its
// gradient with respect to the charges.
//   E = 1/2 q^T A~ q,   dE/dq = 1/2 (A~ + A~^T) q.
// A~ is the HODLR3D operator of Alg. 2; it is not exactly symmetric (Alg. 1
// compresses every ordered pair of boxes on its own), so the gradient takes
// both products.  The quadratic form is reduced in FP64 in a fixed order
// (per-block partial sums, then one block over the partials), so E is
// reproducible run to run.
#include "h3d_internal.cuh"

namespace h3d {
namespace {

constexpr int kEnergyThreads = 256;
constexpr int kEnergyBlocks = 1024;   // partial sums

template <class T>
__global__ void __launch_bounds__(kEnergyThreads) k_energy_partial(const T *__restrict__ q, const T *__restrict__ y,
                                                                   const T *__restrict__ yT, T *__restrict__ grad,
                                                                   int64_t n, double *__restrict__ part) {
    __shared__ double red[kEnergyThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kEnergyThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kEnergyThreads) {
        acc += (double)q[i] * (double)y[i];
        if (grad) grad[i] = (T)(0.5 * ((double)y[i] + (double)yT[i]));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kEnergyThreads) k_energy_final(const double *__restrict__ part, int np,
                                                                 double *__restrict__ E) {
    __shared__ double red[kEnergyThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += kEnergyThreads) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = 0.5 * red[0];
}

}  // namespace

void energy(Handle &h, const void *q, double *E, void *grad, cudaStream_t s) {
    const size_t es = h.elem();
    if (!h.ey) {   // scratch kept by the handle: A~ q, A~^T q, partial sums
        H3D_CUDA(cudaStreamSynchronize(s));
        alloc_all(h.mem, {{&h.ey, (size_t)std::max<int64_t>(h.N, 4) * es},
                          {&h.eyT, (size_t)std::max<int64_t>(h.N, 4) * es},
                          {(void **)&h.epart, kEnergyBlocks * sizeof(double)}});
    }
    run_matvec(h, q, h.ey, 1, false, s);
    // symmetric storage: A~^T q = A~ q, no second product
    if (grad && !h.symmetric()) run_matvec(h, q, h.eyT, 1, true, s);
    const void *yT = grad && h.symmetric() ? h.ey : h.eyT;
    const int nb = (int)std::min<int64_t>(kEnergyBlocks, (h.N + kEnergyThreads - 1) / kEnergyThreads);
    if (h.prec == H3D_FP64)
        k_energy_partial<double><<<nb, kEnergyThreads, 0, s>>>((const double *)q, (const double *)h.ey,
                                                                (const double *)yT, (double *)grad, h.N,
                                                                h.epart);
    else
        k_energy_partial<float><<<nb, kEnergyThreads, 0, s>>>((const float *)q, (const float *)h.ey,
                                                               (const float *)yT, (float *)grad, h.N, h.epart);
    k_energy_final<<<1, kEnergyThreads, 0, s>>>(h.epart, nb, E);
    H3D_LAUNCH_CHECK();
}

}  // namespace h3d

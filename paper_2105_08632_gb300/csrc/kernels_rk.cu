// Elementwise kernels of the RK54 integrator (five-stage fourth-order
// two-register scheme of Carpenter and Kennedy, with an embedded estimate;
// the paper runs its Taylor-Green vortex with it, Sec. 5.3):
//   k_rk2n      per stage i, from the stage's residual R:
//                 dU <- A_i dU + dt R,  U <- U + B_i dU,
//                 E  <- (i == 0 ? 0 : E) + n_i dt R   (optional estimate)
//   k_err_linf  per-CTA maxima of |E| / (atol + rtol max(|U0|, |U|)) (the
//               L-infinity error norm of the paper's adaptive runs).
#include <cstdint>

#include <cuda_runtime.h>

namespace sdrt {

template <typename T>
__global__ void k_rk2n(int64_t n, T* __restrict__ U, T* __restrict__ dU, const T* __restrict__ R, T* __restrict__ E,
                       T a, T b, T ne, T dt, int first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T k = dt * R[i];
        const T d = first ? k : fma(a, dU[i], k);
        dU[i] = d;
        U[i] = fma(b, d, U[i]);
        if (E) E[i] = first ? ne * k : fma(ne, k, E[i]);
    }
}

template <typename T>
__global__ void k_err_linf(int64_t n, const T* __restrict__ E, const T* __restrict__ U0, const T* __restrict__ U,
                           double atol, double rtol, double* __restrict__ part) {
    __shared__ double red[256];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double sc = atol + rtol * fmax(fabs((double)U0[i]), fabs((double)U[i]));
        const double r = fabs((double)E[i]) / sc;
        m = (r > m || r != r) ? r : m;           // a NaN estimate propagates
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = red[threadIdx.x + s];
            if (o > red[threadIdx.x] || o != o) red[threadIdx.x] = o;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <typename T>
void launch_rk2n(int64_t n, T* U, T* dU, const T* R, T* E, double a, double b, double ne, double dt, bool first,
                 int nsm, cudaStream_t st) {
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 8 * (int64_t)nsm ? blocks : 8 * (int64_t)nsm);
    k_rk2n<T><<<grid, 256, 0, st>>>(n, U, dU, R, E, (T)a, (T)b, (T)ne, (T)dt, first ? 1 : 0);
}

template <typename T>
void launch_err_linf(int64_t n, const T* E, const T* U0, const T* U, double atol, double rtol, double* part, int nparts,
                     cudaStream_t st) {
    k_err_linf<T><<<nparts, 256, 0, st>>>(n, E, U0, U, atol, rtol, part);
}

template void launch_rk2n<float>(int64_t, float*, float*, const float*, float*, double, double, double, double, bool,
                                 int, cudaStream_t);
template void launch_rk2n<double>(int64_t, double*, double*, const double*, double*, double, double, double, double,
                                  bool, int, cudaStream_t);
template void launch_err_linf<float>(int64_t, const float*, const float*, const float*, double, double, double*, int,
                                     cudaStream_t);
template void launch_err_linf<double>(int64_t, const double*, const double*, const double*, double, double, double*,
                                      int, cudaStream_t);

}  // namespace sdrt

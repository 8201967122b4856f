// Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt on the device.
//
// Used by every Coulomb-type integral (nuclear attraction and the shell-quartet
// ERIs of the paper's iteration 0, Section 3.1).  Evaluation:
//  * T below a switch point: Taylor expansion of F_L about the nearest table
//    node T_i = i h,  F_L(T_i + d) = sum_k F_{L+k}(T_i) (-d)^k / k!,  then the
//    downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1) (stable);
//  * above it: F_0 = (1/2) sqrt(pi/T) (erf(sqrt T) = 1 to below rounding there)
//    and the upward recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T).
// The table itself is filled once per context by boys_table_kernel from the
// convergent series F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)).
#pragma once
#include "common.cuh"

template <typename T> struct BoysCfg;
template <> struct BoysCfg<double> {
    static constexpr int ncol = BOYS_COL64;
    static constexpr int nterm = 7;
    static constexpr double tmax = BOYS_TMAX64;
};
template <> struct BoysCfg<float> {
    static constexpr int ncol = BOYS_COL32;
    static constexpr int nterm = 4;
    static constexpr double tmax = BOYS_TMAX32;
};

__host__ __device__ __forceinline__ double dev_exp(double x) { return exp(x); }
__host__ __device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__host__ __device__ __forceinline__ double dev_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float dev_sqrt(float x) { return sqrtf(x); }
// read-only load (texture path on the device, plain load when compiled for the host)
template <typename T> __host__ __device__ __forceinline__ T ldg_(const T *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// F[0..L] at T.  tab: row-major [n][ncol] table for this precision.
template <typename T, int L>
__host__ __device__ __forceinline__ void boys_eval(T Targ, const T *__restrict__ tab, T *F) {
    constexpr int NC = BoysCfg<T>::ncol;
    constexpr int NT = BoysCfg<T>::nterm;
    const T tmax = (T)BoysCfg<T>::tmax;
    T ex = dev_exp(-Targ);
    if (Targ < tmax) {
        int i = (int)(Targ * (T)(1.0 / BOYS_H) + (T)0.5);
        T d = Targ - (T)i * (T)BOYS_H;
        const T *row = tab + i * NC + L;
        // Horner: sum_k row[k] (-d)^k / k!
        T acc = ldg_(row + NT - 1);
#pragma unroll
        for (int k = NT - 1; k >= 1; k--) acc = ldg_(row + k - 1) - d * acc / (T)k;
        F[L] = acc;
#pragma unroll
        for (int m = L - 1; m >= 0; m--) F[m] = ((T)2 * Targ * F[m + 1] + ex) / (T)(2 * m + 1);
    } else {
        T rt = (T)1 / dev_sqrt(Targ);
        F[0] = (T)0.88622692545275801365 * rt;  // sqrt(pi)/2 / sqrt(T)
        T o2t = (T)0.5 / Targ;
#pragma unroll
        for (int m = 0; m < L; m++) F[m + 1] = ((T)(2 * m + 1) * F[m] - ex) * o2t;
    }
}

// Generated by gen_dft_consts.py: cos and sin of 2 pi k / R, k < R, for the
// odd radices of the mixed-radix FFT (fft_mr.cuh).
#pragma once

namespace s2g {

template <int R> struct DftConst;
template <> struct DftConst<3> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[3] = {1.000000000e+00f, -5.000000000e-01f, -5.000000000e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[3] = {0.000000000e+00f, 8.660254038e-01f, -8.660254038e-01f};
        return v[k];
    }
};
template <> struct DftConst<5> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[5] = {1.000000000e+00f, 3.090169944e-01f, -8.090169944e-01f, -8.090169944e-01f, 3.090169944e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[5] = {0.000000000e+00f, 9.510565163e-01f, 5.877852523e-01f, -5.877852523e-01f, -9.510565163e-01f};
        return v[k];
    }
};
template <> struct DftConst<7> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[7] = {1.000000000e+00f, 6.234898019e-01f, -2.225209340e-01f, -9.009688679e-01f, -9.009688679e-01f, -2.225209340e-01f, 6.234898019e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[7] = {0.000000000e+00f, 7.818314825e-01f, 9.749279122e-01f, 4.338837391e-01f, -4.338837391e-01f, -9.749279122e-01f, -7.818314825e-01f};
        return v[k];
    }
};
template <> struct DftConst<9> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[9] = {1.000000000e+00f, 7.660444431e-01f, 1.736481777e-01f, -5.000000000e-01f, -9.396926208e-01f, -9.396926208e-01f, -5.000000000e-01f, 1.736481777e-01f, 7.660444431e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[9] = {0.000000000e+00f, 6.427876097e-01f, 9.848077530e-01f, 8.660254038e-01f, 3.420201433e-01f, -3.420201433e-01f, -8.660254038e-01f, -9.848077530e-01f, -6.427876097e-01f};
        return v[k];
    }
};
template <> struct DftConst<11> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[11] = {1.000000000e+00f, 8.412535328e-01f, 4.154150130e-01f, -1.423148383e-01f, -6.548607339e-01f, -9.594929736e-01f, -9.594929736e-01f, -6.548607339e-01f, -1.423148383e-01f, 4.154150130e-01f, 8.412535328e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[11] = {0.000000000e+00f, 5.406408175e-01f, 9.096319954e-01f, 9.898214419e-01f, 7.557495744e-01f, 2.817325568e-01f, -2.817325568e-01f, -7.557495744e-01f, -9.898214419e-01f, -9.096319954e-01f, -5.406408175e-01f};
        return v[k];
    }
};
template <> struct DftConst<13> {
    __host__ __device__ static constexpr float c(int k)
    {
        constexpr float v[13] = {1.000000000e+00f, 8.854560257e-01f, 5.680647467e-01f, 1.205366803e-01f, -3.546048870e-01f, -7.485107482e-01f, -9.709418174e-01f, -9.709418174e-01f, -7.485107482e-01f, -3.546048870e-01f, 1.205366803e-01f, 5.680647467e-01f, 8.854560257e-01f};
        return v[k];
    }
    __host__ __device__ static constexpr float s(int k)
    {
        constexpr float v[13] = {0.000000000e+00f, 4.647231720e-01f, 8.229838659e-01f, 9.927088741e-01f, 9.350162427e-01f, 6.631226582e-01f, 2.393156643e-01f, -2.393156643e-01f, -6.631226582e-01f, -9.350162427e-01f, -9.927088741e-01f, -8.229838659e-01f, -4.647231720e-01f};
        return v[k];
    }
};

}  // namespace s2g

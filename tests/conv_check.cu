// Bitwise check of the integer-pipe conversions in ens_bits.cuh against the hardware
// conversions, and of the bit-split state (split, then join) against its definition, over
// edge cases and pseudo-random bit patterns. Exit code 0 = all agree.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "../paper_2101_09059_gb300/csrc/ens_bits.cuh"

__global__ void conv(const float *xf, const double *xd, int n, double *o64, double *r64,
                     float *o32, float *r32, float *head, double *joined, int *in_range,
                     double *ftz) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    o64[i] = ens::f32_to_f64(xf[i]);
    ftz[i] = ens::f32_to_f64_ftz(xf[i]);
    r64[i] = (double)xf[i];
    o32[i] = ens::f64_to_f32_rz(xd[i]);
    r32[i] = __double2float_rz(xd[i]);
    uint32_t tail;
    in_range[i] = ens::split_state(xd[i], head[i], tail);
    joined[i] = ens::join_state(head[i], tail);
}

int main() {
    const int n = 1 << 22;
    std::vector<float> xf(n);
    std::vector<double> xd(n);
    uint64_t s = 0x9E3779B97F4A7C15ull;
    auto next = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    const float ef[] = {0.0f, -0.0f, 1.0f, -1.0f, 1e-38f, 1.17549435e-38f, 1e-45f, 3.4e38f,
                        __builtin_inff(), -__builtin_inff(), __builtin_nanf("")};
    const double ed[] = {0.0, -0.0, 1.0, -1.0, 1e-38, 1.1754943508222875e-38, 1.1754942e-38,
                         3.4028234663852886e38, 3.5e38, 1e-300, 5e-324, 1e300,
                         __builtin_inf(), -__builtin_inf(), __builtin_nan(""),
                         3.4028236692093846e38, 3.4028236692093841e38, -3.4028236692093841e38,
                         1.0000000000000002, -2.2250738585072014e-308, 1.1754943508222878e-38};
    for (int i = 0; i < n; i++) {
        uint32_t b = (uint32_t)next();
        uint64_t d = next();
        memcpy(&xf[i], &b, 4);
        memcpy(&xd[i], &d, 8);
        if (i % 4 == 1) xd[i] = (double)xf[i] * 1.0000001;         // near float range
        if (i % 4 == 2) xd[i] = ((double)(b % 100000) - 5e4) * 1e-9; // displacements
    }
    for (size_t k = 0; k < sizeof(ef) / 4; k++) xf[k] = ef[k];
    for (size_t k = 0; k < sizeof(ed) / 8; k++) xd[k] = ed[k];
    float *dxf, *do32, *dr32, *dhead;
    double *dxd, *do64, *dr64, *djoin;
    int *drange;
    double *dftz;
    cudaMalloc(&dftz, 8 * n);
    cudaMalloc(&dxf, 4 * n); cudaMalloc(&do32, 4 * n); cudaMalloc(&dr32, 4 * n);
    cudaMalloc(&dxd, 8 * n); cudaMalloc(&do64, 8 * n); cudaMalloc(&dr64, 8 * n);
    cudaMalloc(&dhead, 4 * n); cudaMalloc(&djoin, 8 * n); cudaMalloc(&drange, 4 * n);
    cudaMemcpy(dxf, xf.data(), 4 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dxd, xd.data(), 8 * n, cudaMemcpyHostToDevice);
    conv<<<(n + 255) / 256, 256>>>(dxf, dxd, n, do64, dr64, do32, dr32, dhead, djoin, drange, dftz);
    std::vector<double> o64(n), r64(n), joined(n);
    std::vector<float> o32(n), r32(n), head(n);
    std::vector<int> in_range(n);
    std::vector<double> ftz(n);
    cudaMemcpy(o64.data(), do64, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(r64.data(), dr64, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(o32.data(), do32, 4 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(r32.data(), dr32, 4 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(head.data(), dhead, 4 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(joined.data(), djoin, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(in_range.data(), drange, 4 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(ftz.data(), dftz, 8 * n, cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) { printf("cuda error\n"); return 2; }
    long bad64 = 0, bad32 = 0, flushed = 0;
    for (int i = 0; i < n; i++) {
        if (memcmp(&o64[i], &r64[i], 8) != 0 && !(o64[i] != o64[i] && r64[i] != r64[i])) bad64++;
        // NaN must stay NaN in both directions
        if ((xf[i] != xf[i]) != (o64[i] != o64[i])) bad64++;
        if ((xd[i] != xd[i]) != (o32[i] != o32[i])) bad32++;
        const double ad = xd[i] < 0 ? -xd[i] : xd[i];
        if (ad < 1.1754943508222875e-38) {   // below the binary32 normal range: signed zero
            uint32_t ob; memcpy(&ob, &o32[i], 4);
            uint64_t db; memcpy(&db, &xd[i], 8);
            if ((ob & 0x7fffffffu) != 0 || (ob >> 31) != (uint32_t)(db >> 63)) bad32++;
            flushed++;
        } else if (memcmp(&o32[i], &r32[i], 4) != 0 && !(o32[i] != o32[i] && r32[i] != r32[i])) {
            bad32++;
        }
    }
    // bit-split state: in range <=> |x| < 2^128; there the head is the truncation toward
    // zero (signed zero below 2^-126) and head + tail rebuild x exactly (signed zero below
    // 2^-126)
    long bad_split = 0, split_exact = 0;
    for (int i = 0; i < n; i++) {
        const double ad = xd[i] < 0 ? -xd[i] : xd[i];
        const bool want = ad < 3.4028236692093846e38;  // 2^128; false for NaN
        if ((in_range[i] != 0) != want) { bad_split++; continue; }
        if (!want) continue;
        uint64_t db, jb; uint32_t hb, rb;
        memcpy(&db, &xd[i], 8); memcpy(&jb, &joined[i], 8);
        memcpy(&hb, &head[i], 4); memcpy(&rb, &o32[i], 4);
        if (hb != rb) bad_split++;  // same truncation as f64_to_f32_rz
        if (ad < 1.1754943508222875e-38) {
            if (jb != (db & 0x8000000000000000ull)) bad_split++;
        } else if (jb != db) {
            bad_split++;
        } else {
            split_exact++;
        }
    }
    // flush-to-zero form: exact for normal values and zeros, signed zero for subnormals,
    // a finite magnitude >= 2^128 for Inf and NaN
    long bad_ftz = 0;
    for (int i = 0; i < n; i++) {
        uint32_t b; memcpy(&b, &xf[i], 4);
        const uint32_t e = (b >> 23) & 0xffu;
        uint64_t fb, rb; memcpy(&fb, &ftz[i], 8); memcpy(&rb, &r64[i], 8);
        if (e == 0xffu) {
            const double a = ftz[i] < 0 ? -ftz[i] : ftz[i];
            if (!(a >= 3.4028236692093846e38 && a < 1e300)) bad_ftz++;
        } else if (e == 0u) {
            if (fb != (uint64_t)(b >> 31) << 63) bad_ftz++;
        } else if (fb != rb) {
            bad_ftz++;
        }
    }
    printf("f32->f64 (flush-to-zero form) mismatches %ld\n", bad_ftz);
    bad64 += bad_ftz;
    printf("f32->f64 mismatches %ld, f64->f32 mismatches %ld (of %d; %ld below the normal range)\n",
           bad64, bad32, n, flushed);
    printf("split/join mismatches %ld (%ld values rebuilt exactly)\n", bad_split, split_exact);
    return (bad64 || bad32 || bad_split) ? 1 : 0;
}

// pack.cuh -- conversion of the FP64 master theta into the packed,
// kernel-friendly weight layout (PackOff) in the recurrence precision.
#pragma once
#include "common.cuh"

namespace nqs {

template <typename T>
__global__ void k_pack(const double *__restrict__ th, T *__restrict__ pk, Layout L, PackOff P) {
  const int dh = L.dh, din = L.din, w = dh + din;
  const int64_t tot = P.total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (e >= P.WgT && e < P.WgT + (int64_t)dh * 3 * dh) {
      int64_t q = e - P.WgT; int k = q / (3 * dh), n = q % (3 * dh), a = n / 3, g = n % 3;
      int64_t base = g == 0 ? L.Wu : (g == 1 ? L.Wr : L.Wh);
      v = th[base + (int64_t)a * (g == 2 ? dh : w) + k];
    } else if (e >= P.Wg && e < P.Wg + (int64_t)3 * dh * dh) {
      int64_t q = e - P.Wg; int n = q / dh, b = q % dh, a = n / 3, g = n % 3;
      int64_t base = g == 0 ? L.Wu : (g == 1 ? L.Wr : L.Wh);
      v = th[base + (int64_t)a * (g == 2 ? dh : w) + b];
    } else if (e >= P.xw && e < P.xw + (int64_t)din * 3 * dh) {
      int64_t q = e - P.xw; int d = q / (3 * dh), n = q % (3 * dh), a = n / 3, g = n % 3;
      v = g == 0 ? th[L.Wu + (int64_t)a * w + dh + d]
        : (g == 1 ? th[L.Wr + (int64_t)a * w + dh + d] : th[L.Win + (int64_t)a * din + d]);
    } else if (e >= P.bias && e < P.bias + (int64_t)dh * 4) {
      int64_t q = e - P.bias; int a = q / 4, g = q % 4;
      v = th[(g == 0 ? L.bu : g == 1 ? L.br : g == 2 ? L.bh : L.bin) + a];
    } else if (e >= P.head && e < P.head + 4 * dh) {
      int64_t q = e - P.head; int o = q / dh, b = q % dh;
      v = o < 2 ? th[L.Uo + o * dh + b] : (L.cplx ? th[L.Up + (o - 2) * dh + b] : 0.0);
    } else if (e >= P.hc && e < P.hc + 4) {
      int o = e - P.hc;
      v = o < 2 ? th[L.co + o] : (L.cplx ? th[L.cp + o - 2] : 0.0);
    } else if (L.dim == 2 && e >= P.U12T && e < P.U12T + (int64_t)2 * dh * dh) {
      int64_t q = e - P.U12T; int k = q / dh, a = q % dh;
      v = k < dh ? th[L.U1 + (int64_t)a * dh + k] : th[L.U2 + (int64_t)a * dh + (k - dh)];
    } else if (L.dim == 2 && e >= P.U12 && e < P.U12 + (int64_t)2 * dh * dh) {
      int64_t q = e - P.U12; int a = q / (2 * dh), b = q % (2 * dh);
      v = b < dh ? th[L.U1 + (int64_t)a * dh + b] : th[L.U2 + (int64_t)a * dh + (b - dh)];
    }
    pk[e] = (T)v;
  }
}

}  // namespace nqs

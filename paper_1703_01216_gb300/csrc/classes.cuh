// Frequency classes of the half spectrum (internal): class c = (p, q) with p >= q >= 0 indexes the
// bins (kx, ky) equal up to the sampled kernel's 8-fold symmetry (k -> -k per axis, kx <-> ky), and
// their member bins in the stored half spectrum [kx in 0..n/2][ky in 0..n-1].
#pragma once

namespace fr3d {

__device__ inline void class_pq_m(int c, int& p, int& q) {
  p = (int)((sqrtf(8.f * (float)c + 1.f) - 1.f) * 0.5f);
  while ((p + 1) * (p + 2) / 2 <= c) ++p;
  while (p * (p + 1) / 2 > c) --p;
  q = c - p * (p + 1) / 2;
}

// members (kx, ky) of class c in the stored half spectrum and their weights (1 on the kx = 0 and
// kx = n/2 rows, whose mirror bins are stored too, 2 elsewhere)
__device__ inline int class_members(int c, int n, int* kxs, int* kys, float* wts) {
  int p, q, nm = 0;
  class_pq_m(c, p, q);
  kxs[nm] = p; kys[nm++] = q;
  if (q != 0 && 2 * q != n) { kxs[nm] = p; kys[nm++] = n - q; }
  if (p != q) {
    kxs[nm] = q; kys[nm++] = p;
    if (p != 0 && 2 * p != n) { kxs[nm] = q; kys[nm++] = n - p; }
  }
  for (int m = 0; m < nm; ++m) wts[m] = (kxs[m] == 0 || 2 * kxs[m] == n) ? 1.f : 2.f;
  return nm;
}

}  // namespace fr3d

// View-dependent colour by spherical harmonics (Sec. II-A: Gaussian splatting models colour
// with spherical harmonics; GS-SLAM variants drop them, Sec. II-B).
//
// A Gaussian holds (D + 1)^2 RGB coefficient triples f_i (degree D = 0..3), ordered by band l
// and m = -l..l. The basis is the real spherical harmonics with the Condon-Shortley phase,
// each written as its polynomial in the unit direction u = (x, y, z) from the camera centre
// C = -R^T t to the Gaussian mean; colour = max(sum_i Y_i(u) f_i + 1/2, 0) per channel.
// Shared by the projection (forward, per view) and its backward.
#pragma once

#include "gs_internal.cuh"

namespace gs {

// normalisation constants (closed forms): 1/(2 sqrt(pi)); sqrt(3/(4 pi)); sqrt(15/pi)/2;
// sqrt(5/pi)/4; sqrt(15/pi)/4; sqrt(35/(2 pi))/4; sqrt(105/pi)/2; sqrt(21/(2 pi))/4;
// sqrt(7/pi)/4; sqrt(105/pi)/4
constexpr float kShC0 = 0.28209479177387814f;
constexpr float kShC1 = 0.4886025119029199f;
constexpr float kShC2A = 1.0925484305920792f;
constexpr float kShC2B = 0.31539156525252005f;
constexpr float kShC2C = 0.5462742152960396f;
constexpr float kShC3A = 0.5900435899266435f;
constexpr float kShC3B = 2.890611442640554f;
constexpr float kShC3C = 0.4570457994644658f;
constexpr float kShC3D = 0.3731763325901154f;
constexpr float kShC3E = 1.445305721320277f;
constexpr int kShMaxCoeffs = 16;

// All 16 basis values at the unit vector (x, y, z) (a caller of degree D uses the first (D+1)^2).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float (&Y)[kShMaxCoeffs]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kShC0;
  Y[1] = -kShC1 * y;
  Y[2] = kShC1 * z;
  Y[3] = -kShC1 * x;
  Y[4] = kShC2A * x * y;
  Y[5] = -kShC2A * y * z;
  Y[6] = kShC2B * (2.0f * zz - xx - yy);
  Y[7] = -kShC2A * x * z;
  Y[8] = kShC2C * (xx - yy);
  Y[9] = -kShC3A * y * (3.0f * xx - yy);
  Y[10] = kShC3B * x * y * z;
  Y[11] = -kShC3C * y * (4.0f * zz - xx - yy);
  Y[12] = kShC3D * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -kShC3C * x * (4.0f * zz - xx - yy);
  Y[14] = kShC3E * z * (xx - yy);
  Y[15] = -kShC3A * x * (xx - 3.0f * yy);
}

// (gx, gy, gz) = sum_i s_i grad Y_i at (x, y, z), the gradient of each polynomial above
// (entries of s past the caller's (D+1)^2 must be zero).
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float (&s)[kShMaxCoeffs], float& gx,
                                             float& gy, float& gz) {
  const float xx = x * x, yy = y * y, zz = z * z;
  gx = 0.0f, gy = 0.0f, gz = 0.0f;
  // band 1
  gy -= kShC1 * s[1];
  gz += kShC1 * s[2];
  gx -= kShC1 * s[3];
  // band 2
  gx += kShC2A * y * s[4];
  gy += kShC2A * x * s[4];
  gy -= kShC2A * z * s[5];
  gz -= kShC2A * y * s[5];
  gx -= 2.0f * kShC2B * x * s[6];
  gy -= 2.0f * kShC2B * y * s[6];
  gz += 4.0f * kShC2B * z * s[6];
  gx -= kShC2A * z * s[7];
  gz -= kShC2A * x * s[7];
  gx += 2.0f * kShC2C * x * s[8];
  gy -= 2.0f * kShC2C * y * s[8];
  // band 3
  gx -= 6.0f * kShC3A * x * y * s[9];
  gy -= 3.0f * kShC3A * (xx - yy) * s[9];
  gx += kShC3B * y * z * s[10];
  gy += kShC3B * x * z * s[10];
  gz += kShC3B * x * y * s[10];
  gx += 2.0f * kShC3C * x * y * s[11];
  gy -= kShC3C * (4.0f * zz - xx - 3.0f * yy) * s[11];
  gz -= 8.0f * kShC3C * y * z * s[11];
  gx -= 6.0f * kShC3D * x * z * s[12];
  gy -= 6.0f * kShC3D * y * z * s[12];
  gz += kShC3D * (6.0f * zz - 3.0f * xx - 3.0f * yy) * s[12];
  gx -= kShC3C * (4.0f * zz - 3.0f * xx - yy) * s[13];
  gy += 2.0f * kShC3C * x * y * s[13];
  gz -= 8.0f * kShC3C * x * z * s[13];
  gx += 2.0f * kShC3E * x * z * s[14];
  gy -= 2.0f * kShC3E * y * z * s[14];
  gz += kShC3E * (xx - yy) * s[14];
  gx -= 3.0f * kShC3A * (xx - yy) * s[15];
  gy += 6.0f * kShC3A * x * y * s[15];
}

// Unit direction from the camera centre C = -R^T t to the mean p; inv_r = 1 / |p - C|
// (0 for a mean at the centre, whose direction is then 0).
struct ShDir {
  float x, y, z, inv_r;
};
__device__ __forceinline__ ShDir sh_dir(float p0, float p1, float p2, const gs_camera_t& cam) {
  const float* R = cam.R;
  const float* t = cam.t;
  const float c0 = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
  const float c1 = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
  const float c2 = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
  const float d0 = p0 - c0, d1 = p1 - c1, d2 = p2 - c2;
  const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
  const float inv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
  return {d0 * inv, d1 * inv, d2 * inv, inv};
}

// Unclamped colour sum_i Y_i f_i + 1/2 of Gaussian g (coefficients [N, nc, 3] in `f` with the
// attribute dtype); `finite` is cleared when a coefficient is not finite.
__device__ __forceinline__ float3 sh_raw(const void* f, int dtype, int64_t g, int nc, const float (&Y)[kShMaxCoeffs],
                                         bool& finite) {
  float3 c = make_float3(0.5f, 0.5f, 0.5f);
  const int64_t base = g * nc * 3;
#pragma unroll
  for (int i = 0; i < kShMaxCoeffs; ++i) {
    if (i < nc) {
      const float a = load_attr(f, base + 3 * i + 0, dtype);
      const float b = load_attr(f, base + 3 * i + 1, dtype);
      const float e = load_attr(f, base + 3 * i + 2, dtype);
      finite = finite && isfinite(a) && isfinite(b) && isfinite(e);
      c.x = fmaf(Y[i], a, c.x);
      c.y = fmaf(Y[i], b, c.y);
      c.z = fmaf(Y[i], e, c.z);
    }
  }
  return c;
}

}  // namespace gs

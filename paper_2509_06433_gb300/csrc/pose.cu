// Pose update of render-based tracking: one Adam step on the se(3) increment of each view's
// camera pose, applied on the left: T <- Exp(xi) T with xi = -(lr * Adam direction).
// The state (first and second moments, step count) lives on the device, so a whole tracking
// iteration can be replayed from a CUDA graph without host round trips.
#include "gs_internal.cuh"

namespace gs {
namespace {

struct M3 {
  float m[3][3];
};

__device__ __forceinline__ M3 skew(const float w[3]) {
  M3 S{};
  S.m[0][1] = -w[2];
  S.m[0][2] = w[1];
  S.m[1][0] = w[2];
  S.m[1][2] = -w[0];
  S.m[2][0] = -w[1];
  S.m[2][1] = w[0];
  return S;
}

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
  return c;
}

__global__ void k_pose_adam(gs_camera_t* __restrict__ cams, float* __restrict__ grad, float* __restrict__ state, int K,
                            float lr_rho, float lr_phi, float b1, float b2, float eps, int zero_grad) {
  pdl_begin();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  float* st = state + 16 * k;
  const float t = st[12] + 1.0f;
  st[12] = t;
  const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
  float xi[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float g = grad[6 * k + i];
    const float m = b1 * st[i] + (1.0f - b1) * g;
    const float v = b2 * st[6 + i] + (1.0f - b2) * g * g;
    st[i] = m;
    st[6 + i] = v;
    const float lr = i < 3 ? lr_rho : lr_phi;
    xi[i] = -lr * (m / c1) / (sqrtf(v / c2) + eps);
    if (zero_grad) grad[6 * k + i] = 0.0f;
  }
  // Exp of se(3): R_phi = I + a [phi]x + b [phi]x^2, V = I + b [phi]x + c [phi]x^2
  const float* phi = xi + 3;
  const float th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  const float th = sqrtf(th2);
  float a, b, c;
  if (th < 1e-4f) {  // series to third order
    a = 1.0f - th2 / 6.0f;
    b = 0.5f - th2 / 24.0f;
    c = 1.0f / 6.0f - th2 / 120.0f;
  } else {
    a = sinf(th) / th;
    b = (1.0f - cosf(th)) / th2;
    c = (th - sinf(th)) / (th2 * th);
  }
  const M3 W = skew(phi);
  const M3 W2 = mul(W, W);
  M3 Rp, V;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float id = i == j ? 1.0f : 0.0f;
      Rp.m[i][j] = id + a * W.m[i][j] + b * W2.m[i][j];
      V.m[i][j] = id + b * W.m[i][j] + c * W2.m[i][j];
    }
  gs_camera_t cam = cams[k];
  M3 R;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R.m[i][j] = cam.R[3 * i + j];
  M3 Rn = mul(Rp, R);
  float tn[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    tn[i] = Rp.m[i][0] * cam.t[0] + Rp.m[i][1] * cam.t[1] + Rp.m[i][2] * cam.t[2] + V.m[i][0] * xi[0] +
            V.m[i][1] * xi[1] + V.m[i][2] * xi[2];
  // re-orthonormalise the rows (Gram-Schmidt) so rounding does not accumulate over iterations
  float r0[3] = {Rn.m[0][0], Rn.m[0][1], Rn.m[0][2]};
  float n0 = rsqrtf(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
  for (int j = 0; j < 3; ++j) r0[j] *= n0;
  float r1[3] = {Rn.m[1][0], Rn.m[1][1], Rn.m[1][2]};
  const float d01 = r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2];
  for (int j = 0; j < 3; ++j) r1[j] -= d01 * r0[j];
  const float n1 = rsqrtf(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
  for (int j = 0; j < 3; ++j) r1[j] *= n1;
  const float r2[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]};
  for (int j = 0; j < 3; ++j) {
    cam.R[j] = r0[j];
    cam.R[3 + j] = r1[j];
    cam.R[6 + j] = r2[j];
    cam.t[j] = tn[j];
  }
  cams[k] = cam;
}

}  // namespace
}  // namespace gs

extern "C" gs_status_t gs_pose_adam_step(gs_camera_t* d_cams, float* d_pose_grad, float* d_state, int32_t K,
                                         float lr_rho, float lr_phi, float beta1, float beta2, float eps,
                                         int32_t zero_grad, void* stream) {
  if (!d_cams || !d_pose_grad || !d_state || K < 1 || K > 1024) return GS_ERR_INVALID_ARG;
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f)) return GS_ERR_INVALID_ARG;
  gs::launch(gs::k_pose_adam, (K + 63) / 64, 64, 0, static_cast<cudaStream_t>(stream), d_cams, d_pose_grad, d_state, K, lr_rho,
                                                                                  lr_phi, beta1, beta2, eps, zero_grad);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

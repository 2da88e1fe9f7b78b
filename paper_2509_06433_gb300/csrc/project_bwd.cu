// Backward of the projection: per Gaussian, sum its per-(view, tile) gradient records in a
// fixed order, then apply the chain rule of the projection to the Gaussian parameters and
// to each view's se(3) pose. One thread per Gaussian loops over the K views, so the
// parameter gradients are accumulated without atomics; pose gradients are reduced per
// block and then across blocks in a fixed order.
//
// Forward (recomputed in FP32): p_c = R p + t; Q = rot(q / |q|); M = Q diag(exp(s));
// Nm = R M; J = [[fx/z, 0, -fx tx/z], [0, fy/z, -fy ty/z]] with tx, ty the clamped x/z, y/z;
// m = J Nm (2x3); Sigma2 = m m^T + 0.3 I; conic X = Sigma2^-1; u = fx x/z + cx, v = fy y/z + cy.
// Reverse: dSigma2 = -X Gbar X, dm = 2 dSigma2 m, dJ = dm Nm^T, dNm = J^T dm, dM = R^T dNm,
// dQ = dM diag(s), ds = diag(Q^T dM), dq through the normalisation; dp_c from J, (u, v), z;
// pose (left perturbation): drho = dp_c, dphi = p_c x dp_c + vee(Nm dNm^T - dNm Nm^T).
#include "gs_internal.cuh"
#include "sh.cuh"

namespace gs {
namespace {

// *p += v, or with `store` *p = v (the old value is not read: it may be uninitialised)
__device__ __forceinline__ void put(float* p, bool store, float v) { *p = store ? v : *p + v; }

struct Sum10 {
  float v[10];
};

// Sums the records of slots [off, off + cnt) whose bit is set in `valid` (the others were
// not written: zero gradient), in increasing slot order, clipped to the workspace capacity
// (pairs past the capacity were never emitted when the pair count overflowed; the error word
// reports that case).
__device__ __forceinline__ void add_record(float (&v)[10], const float* __restrict__ pg, uint32_t slot) {
  const float4* r = reinterpret_cast<const float4*>(pg + static_cast<size_t>(slot) * kPairGradStride);
  const float4 a = r[0], b = r[1], c = r[2];
  v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w;
  v[4] += b.x; v[5] += b.y; v[6] += b.z; v[7] += b.w;
  v[8] += c.x; v[9] += c.y;
}

__device__ __forceinline__ void clip(uint32_t off, uint32_t& cnt, int64_t cap) {
  if (static_cast<int64_t>(off) >= cap) cnt = 0;
  else if (static_cast<int64_t>(off) + cnt > cap) cnt = static_cast<uint32_t>(cap - off);
}

__device__ __forceinline__ Sum10 sum_pairs(const float* __restrict__ pg, const uint32_t* __restrict__ valid,
                                           uint32_t off, uint32_t cnt, int64_t cap) {
  clip(off, cnt, cap);
  Sum10 s;
#pragma unroll
  for (int i = 0; i < 10; ++i) s.v[i] = 0.0f;
  // groups of 4 slots: the marked records' loads are independent (predicated), so they are in
  // flight together; unmarked slots load nothing
  uint32_t wi = 0xffffffffu, word = 0;
  for (uint32_t j = 0; j < cnt; j += 4) {
    float4 a[4], b[4], c[4];
    bool on[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t slot = off + j + q;
      if ((slot >> 5) != wi) {
        wi = slot >> 5;
        word = valid[wi];
      }
      on[q] = (j + q < cnt) && ((word >> (slot & 31)) & 1u);
      a[q] = b[q] = c[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (on[q]) {
        const float4* r = reinterpret_cast<const float4*>(pg + static_cast<size_t>(slot) * kPairGradStride);
        a[q] = r[0];
        b[q] = r[1];
        c[q] = r[2];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!on[q]) continue;
      s.v[0] += a[q].x; s.v[1] += a[q].y; s.v[2] += a[q].z; s.v[3] += a[q].w;
      s.v[4] += b[q].x; s.v[5] += b[q].y; s.v[6] += b[q].z; s.v[7] += b[q].w;
      s.v[8] += c[q].x; s.v[9] += c[q].y;
    }
  }
  return s;
}

// Warp-wide version: a lane whose item has more than kCoopPairs records gets them summed
// by the whole warp (lane-strided partial sums, then a fixed butterfly), the others sum
// their own serially. Every lane of the warp must call it. Deterministic.
constexpr uint32_t kCoopPairs = 32;
__device__ __forceinline__ Sum10 sum_pairs_warp(const float* __restrict__ pg, const uint32_t* __restrict__ valid,
                                                uint32_t off, uint32_t cnt, int64_t cap, bool active) {
  const int lane = threadIdx.x & 31;
  if (!active) cnt = 0;
  const bool big = cnt > kCoopPairs;
  Sum10 mine = sum_pairs(pg, valid, off, big ? 0u : cnt, cap);
  uint32_t pending = __ballot_sync(0xffffffffu, big);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const uint32_t o = __shfl_sync(0xffffffffu, off, src);
    uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
    clip(o, c, cap);
    Sum10 part;
#pragma unroll
    for (int i = 0; i < 10; ++i) part.v[i] = 0.0f;
    for (uint32_t j = lane; j < c; j += 32) {
      const uint32_t slot = o + j;
      if ((valid[slot >> 5] >> (slot & 31)) & 1u) add_record(part.v, pg, slot);
    }
#pragma unroll
    for (int i = 0; i < 10; ++i)
#pragma unroll
      for (int x = 16; x > 0; x >>= 1) part.v[i] += __shfl_xor_sync(0xffffffffu, part.v[i], x);
    if (lane == src) mine = part;
  }
  return mine;
}

// Blocks of k_item_grads: up to eight per multiprocessor, no more than there are chunks.
int64_t item_grad_blocks(const Layout& L) {
  const int64_t resident = static_cast<int64_t>(device_sms()) * 8;
  return L.n_item_chunks < resident ? L.n_item_chunks : resident;
}

// Per-item partial gradient of the projection backward (16 floats): the mean's gradient in
// world coordinates (0-2), the gradient of M = Q diag(exp(s)) (3-11, row-major), the opacity's
// (12) and the colour's (13-15; with spherical harmonics the colour gradient after the clamp).
constexpr int kPartial = 16;

// Backward of the projection for one live (view, Gaussian) item, one thread per item in the
// compact order of the live items (increasing k N + g): sums the item's pair records in slot
// order (warp-cooperatively for items with many pairs), applies the chain rule of the view's
// projection, writes the item's partial (when parameter gradients are wanted) and sums the
// items' pose gradients per view. Blocks take chunks of kPoseBlock live items from a counter
// (balanced whatever the chunks' work); a chunk's items are in view order, so each view k present
// in chunk c gets the chunk's sum in slot c + k of pose_partials (unique: a later chunk's first
// view is at least this chunk's last), which k_pose_reduce sums over the view's chunks in order.
__global__ void __launch_bounds__(kPoseBlock, 4) k_item_grads(Layout L, GaussPtrs G, const gs_camera_t* __restrict__ cams,
                                                          uint8_t* __restrict__ ws, int want_params,
                                                          float* __restrict__ pose_partials) {
  pdl_wait();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t n_live = at<Status>(ws, L.status)->n_live;
  const int64_t chunks = (n_live + kPoseBlock - 1) / kPoseBlock;
  const uint32_t* live_kg = at<uint32_t>(ws, L.live_kg);
  const uint32_t* live_off = at<uint32_t>(ws, L.live_off);
  const uint32_t* live_count = at<uint32_t>(ws, L.live_count);
  const float* pg = at<float>(ws, L.pair_grads);
  const uint32_t* pvalid = at<uint32_t>(ws, L.pair_valid);
  float4* partials = at<float4>(ws, L.item_partials);
  __shared__ float s_red[kPoseBlock / 32][6];
  __shared__ int s_k0, s_k1;
  __shared__ int64_t s_chunk;
  uint32_t* ctr = &at<Status>(ws, L.status)->grad_chunk_ctr;
  for (;;) {
    __syncthreads();  // the previous chunk's s_k0 / s_k1 / s_chunk are read
    if (threadIdx.x == 0) s_chunk = atomicAdd(ctr, 1u);
    __syncthreads();
    const int64_t c = s_chunk;
    if (c >= chunks) break;
    const int64_t pos = c * kPoseBlock + threadIdx.x;
    const bool valid = pos < n_live;
    uint32_t kg = 0, off = 0, cnt = 0;
    if (valid) {
      kg = live_kg[pos];
      off = live_off[pos];
      cnt = live_count[pos];
    }
    const int k = static_cast<int>(kg / static_cast<uint32_t>(L.N > 0 ? L.N : 1));
    const int64_t g = static_cast<int64_t>(kg) - static_cast<int64_t>(k) * L.N;
    const Sum10 s = sum_pairs_warp(pg, pvalid, off, cnt, L.cap, valid);
    float pose[6] = {0, 0, 0, 0, 0, 0};
    if (valid) {
      float p[3], ls[3], q[4];
      for (int j = 0; j < 3; ++j) p[j] = load_attr(G.means, 3 * g + j, G.means_dtype);
      for (int j = 0; j < 3; ++j) ls[j] = load_attr(G.log_scales, 3 * g + j, G.dtype);
      for (int j = 0; j < 4; ++j) q[j] = load_attr(G.quats, 4 * g + j, G.dtype);
      const float qlen = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      const float iq = qlen > 0.0f ? 1.0f / qlen : 0.0f;
      const float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
      float Q[3][3];
      Q[0][0] = 1.f - 2.f * (y * y + z * z); Q[0][1] = 2.f * (x * y - w * z); Q[0][2] = 2.f * (x * z + w * y);
      Q[1][0] = 2.f * (x * y + w * z); Q[1][1] = 1.f - 2.f * (x * x + z * z); Q[1][2] = 2.f * (y * z - w * x);
      Q[2][0] = 2.f * (x * z - w * y); Q[2][1] = 2.f * (y * z + w * x); Q[2][2] = 1.f - 2.f * (x * x + y * y);
      const float S[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
      float M[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = Q[i][j] * S[j];
      const float gu = s.v[0], gv = s.v[1], gA = s.v[2], gB = s.v[3], gC = s.v[4], gz = s.v[5];
      const gs_camera_t cam = cams[k];
      const float* R = cam.R;
      float pc[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) pc[i] = R[3 * i] * p[0] + R[3 * i + 1] * p[1] + R[3 * i + 2] * p[2] + cam.t[i];
      float Nm[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Nm[i][j] = R[3 * i] * M[0][j] + R[3 * i + 1] * M[1][j] + R[3 * i + 2] * M[2][j];
      const float iz = 1.0f / pc[2];
      const float limx = 1.3f * (0.5f * static_cast<float>(L.W) / cam.fx);
      const float limy = 1.3f * (0.5f * static_cast<float>(L.H) / cam.fy);
      const float rx = pc[0] * iz, ry = pc[1] * iz;
      const bool clx = (rx < -limx) || (rx > limx), cly = (ry < -limy) || (ry > limy);
      const float txz = fminf(fmaxf(rx, -limx), limx), tyz = fminf(fmaxf(ry, -limy), limy);
      const float J00 = cam.fx * iz, J02 = -J00 * txz, J11 = cam.fy * iz, J12 = -J11 * tyz;
      float m1[3], m2[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        m1[j] = J00 * Nm[0][j] + J02 * Nm[2][j];
        m2[j] = J11 * Nm[1][j] + J12 * Nm[2][j];
      }
      const float aa = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
      const float cc = m2[0] * m2[0] + m2[1] * m2[1] + m2[2] * m2[2];
      const float bb = m1[0] * m2[0] + m1[1] * m2[1] + m1[2] * m2[2];
      const float k0 = m1[1] * m2[2] - m1[2] * m2[1], k1 = m1[2] * m2[0] - m1[0] * m2[2],
                  k2 = m1[0] * m2[1] - m1[1] * m2[0];
      const float det = (k0 * k0 + k1 * k1 + k2 * k2) + 0.3f * (aa + cc) + 0.09f;
      const float idet = 1.0f / det;
      const float A = (cc + 0.3f) * idet, B = -bb * idet, C = (aa + 0.3f) * idet;
      // dSigma2 = -X Gbar X with Gbar = [[gA, gB/2], [gB/2, gC]]
      const float hB = 0.5f * gB;
      const float XG00 = A * gA + B * hB, XG01 = A * hB + B * gC;
      const float XG10 = B * gA + C * hB, XG11 = B * hB + C * gC;
      const float G00 = -(XG00 * A + XG01 * B), G01 = -(XG00 * B + XG01 * C);
      const float G10 = -(XG10 * A + XG11 * B), G11 = -(XG10 * B + XG11 * C);
      float dm1[3], dm2[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dm1[j] = 2.0f * (G00 * m1[j] + G01 * m2[j]);
        dm2[j] = 2.0f * (G10 * m1[j] + G11 * m2[j]);
      }
      const float dJ00 = dm1[0] * Nm[0][0] + dm1[1] * Nm[0][1] + dm1[2] * Nm[0][2];
      const float dJ02 = dm1[0] * Nm[2][0] + dm1[1] * Nm[2][1] + dm1[2] * Nm[2][2];
      const float dJ11 = dm2[0] * Nm[1][0] + dm2[1] * Nm[1][1] + dm2[2] * Nm[1][2];
      const float dJ12 = dm2[0] * Nm[2][0] + dm2[1] * Nm[2][1] + dm2[2] * Nm[2][2];
      float dN[3][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dN[0][j] = J00 * dm1[j];
        dN[1][j] = J11 * dm2[j];
        dN[2][j] = J02 * dm1[j] + J12 * dm2[j];
      }
      // camera-space mean
      const float iz2 = iz * iz;
      float dpc[3];
      dpc[0] = gu * cam.fx * iz;
      dpc[1] = gv * cam.fy * iz;
      dpc[2] = gz - gu * cam.fx * pc[0] * iz2 - gv * cam.fy * pc[1] * iz2;
      dpc[2] += -cam.fx * iz2 * dJ00 - cam.fy * iz2 * dJ11 + cam.fx * txz * iz2 * dJ02 + cam.fy * tyz * iz2 * dJ12;
      if (!clx) {
        dpc[0] += -cam.fx * iz2 * dJ02;
        dpc[2] += cam.fx * pc[0] * iz2 * iz * dJ02;
      }
      if (!cly) {
        dpc[1] += -cam.fy * iz2 * dJ12;
        dpc[2] += cam.fy * pc[1] * iz2 * iz * dJ12;
      }
      float dmean[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) dmean[j] = R[j] * dpc[0] + R[3 + j] * dpc[1] + R[6 + j] * dpc[2];
      // pose: rho = dp_c ; phi = p_c x dp_c + vee(A - A^T), A = Nm dN^T
      float Am[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Am[i][j] = Nm[i][0] * dN[j][0] + Nm[i][1] * dN[j][1] + Nm[i][2] * dN[j][2];
      pose[0] = dpc[0];
      pose[1] = dpc[1];
      pose[2] = dpc[2];
      pose[3] = pc[1] * dpc[2] - pc[2] * dpc[1] + Am[1][2] - Am[2][1];
      pose[4] = pc[2] * dpc[0] - pc[0] * dpc[2] + Am[2][0] - Am[0][2];
      pose[5] = pc[0] * dpc[1] - pc[1] * dpc[0] + Am[0][1] - Am[1][0];
      float gc0 = s.v[7], gc1 = s.v[8], gc2 = s.v[9];
      if (L.color_mode == GS_COLOR_SH) {
        // view-dependent colour: the colour gradient through the clamp (raw < 0: zero); its part
        // through the unit direction u = (p - C) / |p - C| goes to the mean, dL/dp = (I - u u^T)
        // (sum_i (f_i . g) grad Y_i) / |p - C|, and, as the camera centre moves by -R^T rho
        // under the pose perturbation, to rho (dL/drho = R dL/dp)
        const ShDir u = sh_dir(p[0], p[1], p[2], cam);
        float Y[kShMaxCoeffs];
        sh_basis(u.x, u.y, u.z, Y);
        bool fin = true;
        const float3 raw = sh_raw(G.rgb, G.dtype, g, L.sh_coeffs, Y, fin);
        gc0 = raw.x >= 0.0f ? gc0 : 0.0f;
        gc1 = raw.y >= 0.0f ? gc1 : 0.0f;
        gc2 = raw.z >= 0.0f ? gc2 : 0.0f;
        if (L.sh_degree > 0) {
          const int64_t base = g * L.sh_coeffs * 3;
          float sv[kShMaxCoeffs];
#pragma unroll
          for (int i = 0; i < kShMaxCoeffs; ++i) {
            sv[i] = 0.0f;
            if (i < L.sh_coeffs)
              sv[i] = gc0 * load_attr(G.rgb, base + 3 * i + 0, G.dtype) + gc1 * load_attr(G.rgb, base + 3 * i + 1, G.dtype) +
                      gc2 * load_attr(G.rgb, base + 3 * i + 2, G.dtype);
          }
          float gx, gy, gzz;
          sh_basis_vjp(u.x, u.y, u.z, sv, gx, gy, gzz);
          const float ud = gx * u.x + gy * u.y + gzz * u.z;
          const float dd0 = (gx - u.x * ud) * u.inv_r, dd1 = (gy - u.y * ud) * u.inv_r, dd2 = (gzz - u.z * ud) * u.inv_r;
          dmean[0] += dd0;
          dmean[1] += dd1;
          dmean[2] += dd2;
          pose[0] += R[0] * dd0 + R[1] * dd1 + R[2] * dd2;
          pose[1] += R[3] * dd0 + R[4] * dd1 + R[5] * dd2;
          pose[2] += R[6] * dd0 + R[7] * dd1 + R[8] * dd2;
        }
      }
      if (want_params) {
        // dM = R^T dN
        float dM[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) dM[i][j] = R[i] * dN[0][j] + R[3 + i] * dN[1][j] + R[6 + i] * dN[2][j];
        float4* dst = partials + pos * (kPartial / 4);
        dst[0] = make_float4(dmean[0], dmean[1], dmean[2], dM[0][0]);
        dst[1] = make_float4(dM[0][1], dM[0][2], dM[1][0], dM[1][1]);
        dst[2] = make_float4(dM[1][2], dM[2][0], dM[2][1], dM[2][2]);
        dst[3] = make_float4(s.v[6], gc0, gc1, gc2);
      }
    }
    // the block's pose sums per view: its items are in view order, from view s_k0 to s_k1
    if (threadIdx.x == 0) s_k0 = valid ? k : 0;
    const bool last_valid = valid && (threadIdx.x == kPoseBlock - 1 || pos + 1 == n_live);
    if (last_valid) s_k1 = k;
    __syncthreads();
    const int k0 = s_k0, k1 = s_k1;
    for (int kk = k0; kk <= k1; ++kk) {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float v = (valid && k == kk) ? pose[i] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[wib][i] = v;
      }
      __syncthreads();
      if (threadIdx.x < 6) {
        float v = 0.0f;
        for (int wv = 0; wv < kPoseBlock / 32; ++wv) v += s_red[wv][threadIdx.x];
        pose_partials[(c + kk) * 6 + threadIdx.x] = v;
      }
      __syncthreads();
    }
  }
  pdl_trigger();
}

// Parameter gradients, one thread per Gaussian: the partials of its live items summed in view
// order (found by their rank among the live items), then the chain rule through M = Q
// diag(exp(s)) to the log-scales and (through the normalisation) the quaternion, the opacity's
// sigmoid to the logit; with spherical harmonics each view's colour gradient goes to the
// coefficients through that view's basis values. A Gaussian that no view sees gets zero
// gradients (stored with out.overwrite, nothing added otherwise).
__global__ void __launch_bounds__(kPoseBlock) k_gaussian_grads(Layout L, GaussPtrs G, const gs_camera_t* __restrict__ cams,
                                                              const uint8_t* __restrict__ ws, gs_grads_t out) {
  pdl_wait();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kPoseBlock + threadIdx.x;
  if (g >= L.N) return;
  const uint32_t* live_mask = at<uint32_t>(ws, L.live_mask);
  const uint32_t* live_wpre = at<uint32_t>(ws, L.live_wpre);
  const float4* partials = at<float4>(ws, L.item_partials);
  const bool store = out.overwrite != 0;
  const bool sh = L.color_mode == GS_COLOR_SH;
  float acc[kPartial];
#pragma unroll
  for (int i = 0; i < kPartial; ++i) acc[i] = 0.0f;
  bool seen = false, sh_touched = false;
  uint32_t words[4], bases[4];
  float p[3] = {0, 0, 0};
  if (sh && out.rgb) for (int j = 0; j < 3; ++j) p[j] = load_attr(G.means, 3 * g + j, G.means_dtype);
  for (int k = 0; k < L.K; ++k) {
    // the mask words and rank bases of four views at a time are loaded together
    if ((k & 3) == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t kgj = static_cast<int64_t>(k + j) * L.N + g;
        words[j] = k + j < L.K ? live_mask[kgj >> 5] : 0u;
        bases[j] = (words[j] >> (kgj & 31)) & 1u ? live_wpre[kgj >> 5] : 0u;
      }
    }
    const int64_t kg = static_cast<int64_t>(k) * L.N + g;
    const uint32_t word = words[k & 3];
    if (!((word >> (kg & 31)) & 1u)) continue;
    seen = true;
    const uint32_t pos = bases[k & 3] + __popc(word & ((1u << (kg & 31)) - 1u));
    const float4* src = partials + static_cast<int64_t>(pos) * (kPartial / 4);
    const float4 a = src[0], b = src[1], c = src[2], d = src[3];
    const float v[kPartial] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
#pragma unroll
    for (int i = 0; i < kPartial; ++i) acc[i] += v[i];
    if (sh && out.rgb) {  // dL/df_i += Y_i(u_k) g_k for this view's direction
      const ShDir u = sh_dir(p[0], p[1], p[2], cams[k]);
      float Y[kShMaxCoeffs];
      sh_basis(u.x, u.y, u.z, Y);
      const int64_t base = g * L.sh_coeffs * 3;
      const bool first = store && !sh_touched;
      for (int i = 0; i < L.sh_coeffs; ++i) {
        float* o3 = out.rgb + base + 3 * i;
        put(o3 + 0, first, Y[i] * d.y);
        put(o3 + 1, first, Y[i] * d.z);
        put(o3 + 2, first, Y[i] * d.w);
      }
      sh_touched = true;
    }
  }
  if (!seen) {
    if (store) {
      if (out.means) out.means[3 * g] = out.means[3 * g + 1] = out.means[3 * g + 2] = 0.0f;
      if (out.log_scales) out.log_scales[3 * g] = out.log_scales[3 * g + 1] = out.log_scales[3 * g + 2] = 0.0f;
      if (out.quats)
        for (int j = 0; j < 4; ++j) out.quats[4 * g + j] = 0.0f;
      if (out.opacity_logits) out.opacity_logits[g] = 0.0f;
      if (out.rgb) {
        const int cw = sh ? 3 * L.sh_coeffs : 3;
        for (int j = 0; j < cw; ++j) out.rgb[cw * g + j] = 0.0f;
      }
    }
    return;
  }
  float ls[3], q[4];
  for (int j = 0; j < 3; ++j) ls[j] = load_attr(G.log_scales, 3 * g + j, G.dtype);
  for (int j = 0; j < 4; ++j) q[j] = load_attr(G.quats, 4 * g + j, G.dtype);
  const float lg = load_attr(G.logits, g, G.dtype);
  const float qlen = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float iq = qlen > 0.0f ? 1.0f / qlen : 0.0f;
  const float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
  float Q[3][3];
  Q[0][0] = 1.f - 2.f * (y * y + z * z); Q[0][1] = 2.f * (x * y - w * z); Q[0][2] = 2.f * (x * z + w * y);
  Q[1][0] = 2.f * (x * y + w * z); Q[1][1] = 1.f - 2.f * (x * x + z * z); Q[1][2] = 2.f * (y * z - w * x);
  Q[2][0] = 2.f * (x * z - w * y); Q[2][1] = 2.f * (y * z + w * x); Q[2][2] = 1.f - 2.f * (x * x + y * y);
  const float S[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
  // M = Q diag(S): dQ = dM diag(S), dS_j = sum_i dM_ij Q_ij
  float dQ[3][3], dls[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float ds = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float dMij = acc[3 + 3 * i + j];
      dQ[i][j] = dMij * S[j];
      ds += dMij * Q[i][j];
    }
    dls[j] = ds * S[j];
  }
  float dqh[4];
  dqh[0] = 2.f * (-z * dQ[0][1] + y * dQ[0][2] + z * dQ[1][0] - x * dQ[1][2] - y * dQ[2][0] + x * dQ[2][1]);
  dqh[1] = 2.f * (y * dQ[0][1] + z * dQ[0][2] + y * dQ[1][0] - 2.f * x * dQ[1][1] - w * dQ[1][2] + z * dQ[2][0] +
                  w * dQ[2][1] - 2.f * x * dQ[2][2]);
  dqh[2] = 2.f * (-2.f * y * dQ[0][0] + x * dQ[0][1] + w * dQ[0][2] + x * dQ[1][0] + z * dQ[1][2] - w * dQ[2][0] +
                  z * dQ[2][1] - 2.f * y * dQ[2][2]);
  dqh[3] = 2.f * (-2.f * z * dQ[0][0] - w * dQ[0][1] + x * dQ[0][2] + w * dQ[1][0] - 2.f * z * dQ[1][1] +
                  y * dQ[1][2] + x * dQ[2][0] + y * dQ[2][1]);
  const float qd = w * dqh[0] + x * dqh[1] + y * dqh[2] + z * dqh[3];
  const float qh[4] = {w, x, y, z};
  const float o = 1.0f / (1.0f + expf(-lg));
  if (out.means)
    for (int j = 0; j < 3; ++j) put(out.means + 3 * g + j, store, acc[j]);
  if (out.log_scales)
    for (int j = 0; j < 3; ++j) put(out.log_scales + 3 * g + j, store, dls[j]);
  if (out.quats)
    for (int j = 0; j < 4; ++j) put(out.quats + 4 * g + j, store, (dqh[j] - qh[j] * qd) * iq);
  if (out.opacity_logits) put(out.opacity_logits + g, store, acc[12] * o * (1.0f - o));
  if (out.rgb && !sh)
    for (int j = 0; j < 3; ++j) put(out.rgb + 3 * g + j, store, acc[13 + j]);
}

// pose[k][i] += (or, with overwrite, =) the sum over the chunks holding view k's live items of
// their slot c + k of pose_partials, in chunk order.
__global__ void k_pose_reduce(const float* __restrict__ partials, Layout L, const uint8_t* __restrict__ ws,
                              float* __restrict__ pose, int overwrite) {
  pdl_begin();
  const int k = blockIdx.x;
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t* mask = at<uint32_t>(ws, L.live_mask);
  const uint32_t* wpre = at<uint32_t>(ws, L.live_wpre);
  const int64_t n_live = at<Status>(ws, L.status)->n_live;
  // the view's live items are positions [r0, r1) among the live items
  auto rank = [&](int64_t item) -> int64_t {
    if (item >= L.KN) return n_live;
    return wpre[item >> 5] + __popc(mask[item >> 5] & ((1u << (item & 31)) - 1u));
  };
  const int64_t r0 = rank(static_cast<int64_t>(k) * L.N), r1 = rank(static_cast<int64_t>(k + 1) * L.N);
  float v = 0.0f;
  if (r1 > r0)
    for (int64_t c = r0 / kPoseBlock + lane; c <= (r1 - 1) / kPoseBlock; c += 32) v += partials[(c + k) * 6 + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) pose[k * 6 + i] = overwrite ? v : pose[k * 6 + i] + v;
}

__global__ void __launch_bounds__(kPoseBlock) k_screen_grads(Layout L, const uint8_t* __restrict__ ws, float* d_mean2d,
                                                            float* d_conic, float* d_depth, float* d_opacity,
                                                            float* d_rgb) {
  pdl_begin();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kPoseBlock + threadIdx.x;
  const bool valid = g < L.N;  // no early return: the pair sums are warp-cooperative
  const uint32_t* live_wpre = at<uint32_t>(ws, L.live_wpre);
  const uint32_t* live_off = at<uint32_t>(ws, L.live_off);
  const uint32_t* live_count = at<uint32_t>(ws, L.live_count);
  const uint32_t* live_mask = at<uint32_t>(ws, L.live_mask);
  const float* pg = at<float>(ws, L.pair_grads);
  const uint32_t* pvalid = at<uint32_t>(ws, L.pair_valid);
  float op = 0.0f, c[3] = {0, 0, 0};
  for (int k = 0; k < L.K; ++k) {
    const int64_t kg = static_cast<int64_t>(k) * L.N + g;
    int4 tl = make_int4(0, 0, 0, 0);  // (pair offset, -, -, tiles emitted)
    if (valid && item_live(live_mask, kg)) {
      const uint32_t pos = live_rank(live_mask, live_wpre, kg);
      tl.x = static_cast<int>(live_off[pos]);
      tl.w = static_cast<int>(live_count[pos]);
    }
    const Sum10 s =
        sum_pairs_warp(pg, pvalid, static_cast<uint32_t>(tl.x), static_cast<uint32_t>(tl.w), L.cap, tl.w > 0);
    if (!valid) continue;
    if (d_mean2d) {
      d_mean2d[2 * kg] = s.v[0];
      d_mean2d[2 * kg + 1] = s.v[1];
    }
    if (d_conic) {
      d_conic[3 * kg] = s.v[2];
      d_conic[3 * kg + 1] = s.v[3];
      d_conic[3 * kg + 2] = s.v[4];
    }
    if (d_depth) d_depth[kg] = s.v[5];
    op += s.v[6];
    c[0] += s.v[7];
    c[1] += s.v[8];
    c[2] += s.v[9];
  }
  if (!valid) return;
  if (d_opacity) d_opacity[g] = op;
  if (d_rgb)
    for (int j = 0; j < 3; ++j) d_rgb[3 * g + j] = c[j];
}

}  // namespace

cudaError_t launch_project_bwd(const Layout& L, const GaussPtrs& g, const gs_camera_t* cams, void* ws,
                               const gs_grads_t& out, cudaStream_t s) {
  if (L.N == 0) {
    if (out.overwrite && out.pose) cudaMemsetAsync(out.pose, 0, sizeof(float) * 6 * L.K, s);
    return cudaGetLastError();
  }
  auto* w = static_cast<uint8_t*>(ws);
  float* partials = at<float>(ws, L.pose_partials);
  const bool params = out.means || out.log_scales || out.quats || out.opacity_logits || out.rgb;
  cudaMemsetAsync(&at<Status>(ws, L.status)->grad_chunk_ctr, 0, sizeof(uint32_t), s);
  launch(k_item_grads, static_cast<unsigned>(item_grad_blocks(L)), kPoseBlock, 0, s, L, g, cams, w, params ? 1 : 0,
         partials);
  if (params) launch(k_gaussian_grads, static_cast<unsigned>(L.n_pose_blocks), kPoseBlock, 0, s, L, g, cams,
                     static_cast<const uint8_t*>(ws), out);
  if (out.pose)
    launch(k_pose_reduce, L.K, 6 * 32, 0, s, static_cast<const float*>(partials), L, static_cast<const uint8_t*>(ws),
           out.pose, out.overwrite);
  return cudaGetLastError();
}

cudaError_t launch_screen_grads(const Layout& L, const void* ws, float* d_mean2d, float* d_conic, float* d_depth,
                                float* d_opacity, float* d_rgb, cudaStream_t s) {
  if (L.N == 0) return cudaSuccess;
  launch(k_screen_grads, static_cast<unsigned>(L.n_pose_blocks), kPoseBlock, 0, s, 
      L, static_cast<const uint8_t*>(ws), d_mean2d, d_conic, d_depth, d_opacity, d_rgb);
  return cudaGetLastError();
}

}  // namespace gs

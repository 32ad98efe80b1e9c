// Derivation (K3f/K4) fused with projection (K5), float32 on CUDA cores.
//
// Per visible anchor of a derivation view (Eq. 3):
//   d = (x_a - p)/|x_a - p|, x = [f_a ; d],
//   h_h = ReLU(W1_h^T x + b1_h) for the opacity, colour and covariance heads,
//   z_h = W2_h^T h_h + b2_h,
//   alpha_j = tanh(z_op[j]) (kept iff > 0), c_j = sigmoid(z_col[3j..]),
//   s_j = s_a sigmoid(z_cov[7j..7j+2]), q_j = normalise(z_cov[7j+3..7j+6]).
// The per-anchor scale and position are broadcast to the k Gaussians inside
// the thread and each attribute goes straight to its consumer (the paper's
// two "combine" operators, Sec. 6, become register moves).  Each kept
// Gaussian is projected at once for every camera this view feeds (EWA,
// Eq. 1-2) and its exact tile count is taken (Sec. 6), so derived
// attributes never round-trip through HBM.
#include "gsc_internal.cuh"

namespace gsc {

constexpr int DER_NT = 128;

struct ProjCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float znear, gx, gy;
  float pc[3], pc_lo[3];
  int W, H;
  uint32_t rec_base;
  uint32_t cam;
};

// EWA projection of one Gaussian + opacity-aware exact tile count.
// Decisions use the pinned depth: mu32 = x_a + o (float32 adds) and
// tz = ((R6 mu_x + R7 mu_y) + R8 mu_z) + t2 without contraction (the order
// the oracle uses for its ordering depth).  The geometry uses camera-relative
// coordinates rel = ((x_a - c_hi) - c_lo) + o, which avoid the cancellation of
// R x + t at city scale.
__device__ __forceinline__ void project_write(const ProjCam& c, Records rec, uint32_t r, const float mu[3],
                                              const float rel[3], float alpha, bool kept, const float col[3],
                                              const float s[3], const float q[4], int TW, int TH) {
  const float tz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], mu[0]), __fmul_rn(c.R[7], mu[1])),
                                       __fmul_rn(c.R[8], mu[2])), c.t[2]);
  float4 geo = make_float4(0.f, 0.f, 0.f, 0.f), cop = make_float4(0.f, 0.f, 0.f, tz);
  uint32_t flag = c.cam;
  uint32_t cnt = 0;
  float4 colv = make_float4(col[0], col[1], col[2], 0.f);
  bool valid = kept && (tz > c.znear) && (alpha >= (1.0f / 255.0f));
  if (valid) {
    const float tx = c.R[0] * rel[0] + c.R[1] * rel[1] + c.R[2] * rel[2];
    const float ty = c.R[3] * rel[0] + c.R[4] * rel[1] + c.R[5] * rel[2];
    const float tza = c.R[6] * rel[0] + c.R[7] * rel[1] + c.R[8] * rel[2];
    const float iz = 1.0f / tza;
    const float txc = fminf(fmaxf(tx * iz, -c.gx), c.gx) * tza;
    const float tyc = fminf(fmaxf(ty * iz, -c.gy), c.gy) * tza;
    const float j00 = c.fx * iz, j02 = -c.fx * txc * iz * iz;
    const float j11 = c.fy * iz, j12 = -c.fy * tyc * iz * iz;
    // T = J W (2x3)
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = j00 * c.R[k] + j02 * c.R[6 + k];
      T1[k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
    }
    // M = R(q) diag(s): Sigma = M M^T
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                   2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                   2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float U0[3], U1[3];  // U = T M
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float m0 = Rq[k] * s[k], m1 = Rq[3 + k] * s[k], m2 = Rq[6 + k] * s[k];
      U0[k] = T0[0] * m0 + T0[1] * m1 + T0[2] * m2;
      U1[k] = T1[0] * m0 + T1[1] * m1 + T1[2] * m2;
    }
    const float a = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2] + 0.3f;
    const float b = U0[0] * U1[0] + U0[1] * U1[1] + U0[2] * U1[2];
    const float cc = U1[0] * U1[0] + U1[1] * U1[1] + U1[2] * U1[2] + 0.3f;
    const float det = a * cc - b * b;
    if (det > 0.f) {
      const float id = 1.0f / det;
      const float A = cc * id, B = -b * id, C = a * id;
      const float mx = c.fx * tx * iz + c.cx, my = c.fy * ty * iz + c.cy;
      const float tau = 2.0f * logf(255.0f * alpha);
      const float tauc = tau * (1.0f + 0.0009765625f) + 0.0009765625f;
      geo = make_float4(mx, my, A, B);
      cop = make_float4(C, alpha, tauc, tz);
      cover_tiles_f32(mx, my, A, B, C, tauc, c.W, c.H, TW, TH, [&](int) { ++cnt; });
      flag |= REC_VALID_BIT;
    }
  }
  colv.w = __uint_as_float(flag);
  rec.geo[r] = geo;
  rec.cop[r] = cop;
  rec.col[r] = colv;
  rec.key[r] = cnt > 0 ? __float_as_uint(tz) : INVALID_KEY;
  rec.cnt[r] = cnt;
}

__global__ void __launch_bounds__(DER_NT) k_derive_f32(const ModelDev* __restrict__ models, int model,
                                                       FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                       Records rec, float* const* __restrict__ dbg_attrs) {
  __shared__ __align__(16) float s_w[W_FLOATS + 2];
  __shared__ int s_d[MAXV];
  __shared__ uint32_t s_b[MAXV + 1];
  __shared__ int s_nd;
  __shared__ ProjCam s_cam[MAXV][2];
  __shared__ float s_pc[MAXV][6];

  const ModelDev md = models[model];
  for (int i = threadIdx.x; i < W_FLOATS; i += DER_NT) s_w[i] = md.w32[i];
  if (threadIdx.x == 0) {
    int nd = 0;
    uint32_t acc = 0;
    for (uint32_t d = 0; d < fd->n_dviews; ++d) {
      if (fd->dcam[d].model != model) continue;
      s_d[nd] = (int)d;
      s_b[nd] = acc;
      acc += fd->vis_count[d];
      for (int u = 0; u < 3; ++u) {
        s_pc[nd][u] = fd->dcam[d].pc[u];
        s_pc[nd][3 + u] = fd->dcam[d].pc_lo[u];
      }
      for (int e = 0; e < 2; ++e) {
        const int ci = fd->dview_cam[d][e];
        ProjCam& pc = s_cam[nd][e];
        pc.cam = ci < 0 ? 0xFFFFFFFFu : (uint32_t)ci;
        if (ci < 0) continue;
        const CamDev& c = fd->cam[ci];
        for (int i = 0; i < 9; ++i) pc.R[i] = c.R[i];
        for (int i = 0; i < 3; ++i) pc.t[i] = c.t[i];
        pc.fx = c.fx; pc.fy = c.fy; pc.cx = c.cx; pc.cy = c.cy;
        pc.znear = c.znear; pc.gx = c.gx; pc.gy = c.gy;
        for (int i = 0; i < 3; ++i) {
          pc.pc[i] = c.pc[i];
          pc.pc_lo[i] = c.pc_lo[i];
        }
        pc.W = c.W; pc.H = c.H;
        pc.rec_base = fd->rec_base[ci];
      }
      ++nd;
    }
    s_b[nd] = acc;
    s_nd = nd;
  }
  __syncthreads();
  const int nd = s_nd;
  const uint32_t total = s_b[nd];
  const uint32_t rec_cap = fd->n_records;
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  int ld = 0;
  for (uint32_t item = blockIdx.x * DER_NT + threadIdx.x; item < total; item += gridDim.x * DER_NT) {
    while (item >= s_b[ld + 1]) ++ld;
    const int d = s_d[ld];
    const uint32_t i = item - s_b[ld];
    const uint32_t a = vis[d][i];
    const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
    // view direction from the derivation camera's double-float centre
    float vx = (xa - s_pc[ld][0]) - s_pc[ld][3];
    float vy = (ya - s_pc[ld][1]) - s_pc[ld][4];
    float vz = (za - s_pc[ld][2]) - s_pc[ld][5];
    const float vn = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
    vx *= vn; vy *= vn; vz *= vn;
    // ---- layer 1 (three heads concatenated): h = ReLU(W1cat^T x + b1cat)
    float h[NH];
#pragma unroll
    for (int o = 0; o < NH; ++o) h[o] = s_w[WOFF_B1 + o];
    const float4* f4 = md.feat + (size_t)a * (FDIM / 4);
#pragma unroll
    for (int c4 = 0; c4 < FDIM / 4; ++c4) {
      const float4 fv = __ldg(f4 + c4);
      const float xs[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4* wr = reinterpret_cast<const float4*>(s_w + WOFF_W1 + (c4 * 4 + u) * NH);
#pragma unroll
        for (int o4 = 0; o4 < NH / 4; ++o4) {
          const float4 w = wr[o4];
          h[4 * o4 + 0] = fmaf(xs[u], w.x, h[4 * o4 + 0]);
          h[4 * o4 + 1] = fmaf(xs[u], w.y, h[4 * o4 + 1]);
          h[4 * o4 + 2] = fmaf(xs[u], w.z, h[4 * o4 + 2]);
          h[4 * o4 + 3] = fmaf(xs[u], w.w, h[4 * o4 + 3]);
        }
      }
    }
    {
      const float xs[3] = {vx, vy, vz};
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const float4* wr = reinterpret_cast<const float4*>(s_w + WOFF_W1 + (FDIM + u) * NH);
#pragma unroll
        for (int o4 = 0; o4 < NH / 4; ++o4) {
          const float4 w = wr[o4];
          h[4 * o4 + 0] = fmaf(xs[u], w.x, h[4 * o4 + 0]);
          h[4 * o4 + 1] = fmaf(xs[u], w.y, h[4 * o4 + 1]);
          h[4 * o4 + 2] = fmaf(xs[u], w.z, h[4 * o4 + 2]);
          h[4 * o4 + 3] = fmaf(xs[u], w.w, h[4 * o4 + 3]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < NH; ++o) h[o] = fmaxf(h[o], 0.f);

    const float sa = __ldg(md.scale + a);
    float* dbg = dbg_attrs ? dbg_attrs[d] : nullptr;
    // ---- layer 2 + activations + projection, one Gaussian at a time
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
      float z[11];
      const int orow[11] = {j, K + 3 * j, K + 3 * j + 1, K + 3 * j + 2, 4 * K + 7 * j, 4 * K + 7 * j + 1,
                            4 * K + 7 * j + 2, 4 * K + 7 * j + 3, 4 * K + 7 * j + 4, 4 * K + 7 * j + 5,
                            4 * K + 7 * j + 6};
#pragma unroll
      for (int u = 0; u < 11; ++u) {
        const int head = u == 0 ? 0 : (u < 4 ? 1 : 2);
        const float4* wr = reinterpret_cast<const float4*>(s_w + WOFF_W2T + orow[u] * HID);
        float acc = s_w[WOFF_B2 + orow[u]];
#pragma unroll
        for (int c4 = 0; c4 < HID / 4; ++c4) {
          const float4 w = wr[c4];
          acc = fmaf(h[head * HID + 4 * c4 + 0], w.x, acc);
          acc = fmaf(h[head * HID + 4 * c4 + 1], w.y, acc);
          acc = fmaf(h[head * HID + 4 * c4 + 2], w.z, acc);
          acc = fmaf(h[head * HID + 4 * c4 + 3], w.w, acc);
        }
        z[u] = acc;
      }
      const float alpha = tanhf(z[0]);
      const bool kept = z[0] > 0.f;
      float col[3], s[3], q[4];
#pragma unroll
      for (int u = 0; u < 3; ++u) col[u] = 1.0f / (1.0f + expf(-z[1 + u]));
#pragma unroll
      for (int u = 0; u < 3; ++u) s[u] = sa * (1.0f / (1.0f + expf(-z[4 + u])));
      const float qn2 = z[7] * z[7] + z[8] * z[8] + z[9] * z[9] + z[10] * z[10];
      if (qn2 < 1e-24f) {
        q[0] = 1.f; q[1] = q[2] = q[3] = 0.f;
      } else {
        const float iq = 1.0f / sqrtf(qn2);
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = z[7 + u] * iq;
      }
      if (dbg) {
        float* o = dbg + ((size_t)i * K + j) * 11;
        o[0] = alpha;
        o[1] = col[0]; o[2] = col[1]; o[3] = col[2];
        o[4] = s[0]; o[5] = s[1]; o[6] = s[2];
        o[7] = q[0]; o[8] = q[1]; o[9] = q[2]; o[10] = q[3];
      }
      const float* op = md.offs + ((size_t)a * K + j) * 3;
      const float o3[3] = {__ldg(op), __ldg(op + 1), __ldg(op + 2)};
      const float mu[3] = {__fadd_rn(xa, o3[0]), __fadd_rn(ya, o3[1]), __fadd_rn(za, o3[2])};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const ProjCam& pc = s_cam[ld][e];
        if (pc.cam == 0xFFFFFFFFu) continue;
        const uint32_t r = pc.rec_base + i * K + (uint32_t)j;
        if (r >= rec_cap) continue;
        const float rel[3] = {((xa - pc.pc[0]) - pc.pc_lo[0]) + o3[0], ((ya - pc.pc[1]) - pc.pc_lo[1]) + o3[1],
                              ((za - pc.pc[2]) - pc.pc_lo[2]) + o3[2]};
        project_write(pc, rec, r, mu, rel, alpha, kept, col, s, q, TW, TH);
      }
    }
  }
}

void launch_derive_f32(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, Records rec,
                       float* const* dbg_attrs, int n_sm, cudaStream_t s) {
  k_derive_f32<<<n_sm * 4, DER_NT, 0, s>>>(models, model, fd, vis, rec, dbg_attrs);
}

}  // namespace gsc

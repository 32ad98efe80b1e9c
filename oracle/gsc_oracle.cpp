// Plain CPU reference ("oracle") of the structured-3DGS per-frame path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code;
// only tests/, __graft_entry__.smoke() and the bench's CPU-baseline leg do.
// It shares no code, header or constant generator with the CUDA library.
//
// Precision: float64 throughout, except the decisions that the method takes
// on floating point and that select discrete sets (visible anchors, the
// near-plane drop, the depth used to order Gaussians).  Those are taken in
// float32 with a fixed operation order ("decision-pinned"), because the CUDA
// path takes them in float32 and an integer decision must be taken in the
// same precision on both sides.  Build with -ffp-contract=off -fno-fast-math.
//
// Paper sections followed (GS-Cache, arXiv 2502.14938):
//   Eq. 1-2 (Sec. 3.1)  Gaussian kernel and covariance R S S^T R^T
//   Eq. 3   (Sec. 3.1)  anchor feature + view direction -> neural Gaussians
//   Sec. 3.1            EWA splatting, tile rasterisation, alpha blending
//   Sec. 3.2 / Alg. 1   anchor filtering (frustum + distance LOD)
//   Eq. 5-6 (Sec. 4)    unified camera for binocular de-redundancy
//   Sec. 6              opacity-aware extent, exact ellipse-tile coverage
// Readings of what the paper leaves open (head layout, activations, LOD rule,
// EWA constants, stop rule, tie order) are listed with the tests that pin
// each function.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct orc_camera {
  float R[9];      // world -> camera rotation, row-major (rows: right, down, forward)
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear;
  int32_t pad;
};

struct orc_model {
  int32_t n, k, n_levels, pad0;
  const float* pos;       // [n][3]
  const float* feat;      // [n][32]
  const float* offs;      // [n][k][3]
  const float* scale;     // [n]
  const uint8_t* level;   // [n]
  float lod_dmax;
  int32_t pad1;
  const float* W1[3];     // [35][32]   (in x out)
  const float* b1[3];     // [32]
  const float* W2[3];     // [32][out_h]
  const float* b2[3];     // [out_h]
  const float* level_offset;  // [n] Octree-GS per-anchor level offsets, or null
  float lod_blend;            // level fade width (applied by the Python layer)
  int32_t pad2;
};

// Quantisation of the decoder MLPs (precision forms).  mode 0: none (fp64);
// 1: bf16 inputs/weights/hidden; 2: fp8-e4m3 with per-tensor scales.
struct orc_quant {
  int32_t mode;
  int32_t pad;
  float s_x;        // fp8 scale of the input vector [f, d]
  float s_h[3];     // fp8 scale of each head's hidden activations
  float s_w1[3];    // fp8 scale of W1 per head
  float s_w2[3];    // fp8 scale of W2 per head
};

}  // extern "C"

namespace {

constexpr int FDIM = 32;
constexpr int IN = 35;
constexpr int HID = 32;

// ---------------------------------------------------------------- rounding
// bf16 round-to-nearest-even of a float32 value (bit definition of bfloat16).
float round_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan unchanged
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// fp8 e4m3 (OCP "E4M3FN": bias 7, max 448, no inf) round-to-nearest-even,
// saturating to +-448.  Written from the format definition.
double round_e4m3(double x) {
  if (std::isnan(x)) return x;
  double a = std::fabs(x);
  if (a >= 448.0) return std::copysign(448.0, x);
  // subnormal spacing 2^-9 below 2^-6; normal spacing 2^(e-3)
  int e;
  std::frexp(a, &e);          // a = m * 2^e, m in [0.5,1)  -> exponent of leading bit is e-1
  int lead = e - 1;
  if (lead < -6) lead = -6;
  double q = std::ldexp(1.0, lead - 3);
  double v = a / q;
  double fl = std::floor(v);
  double fr = v - fl;
  double r;
  if (fr > 0.5) r = fl + 1.0;
  else if (fr < 0.5) r = fl;
  else r = (std::fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
  double out = r * q;
  if (out > 448.0) out = 448.0;
  return std::copysign(out, x);
}

// Two-term E4M3 expansion of v at scale s (a power of two): hi = e4m3(v / s),
// lo = e4m3(v / s - hi), both in units of s (round to nearest even,
// saturating); returns (hi + lo) s and, with hi_out, hi s.  v / s and the
// residual are exact in double.  The FP8 form keeps its weights and hidden
// activations this way: two E4M3 tensors at one per-tensor scale whose sum
// carries about twice the mantissa bits.
double e4m3_two_term(double v, double s, double* hi_out) {
  const double x = v / s;
  const double hi = round_e4m3(x);
  const double lo = round_e4m3(x - hi);
  if (hi_out) *hi_out = hi * s;
  return (hi + lo) * s;
}

// ---------------------------------------------------------------- cameras
void center64(const orc_camera* c, double p[3]) {
  // p = -R^T t, summed in a fixed order
  const float* R = c->R;
  for (int i = 0; i < 3; ++i) {
    double s = (double)R[0 * 3 + i] * (double)c->t[0];
    s = s + (double)R[1 * 3 + i] * (double)c->t[1];
    s = s + (double)R[2 * 3 + i] * (double)c->t[2];
    p[i] = -s;
  }
}

// ---------------------------------------------------------------- sigmoid etc
inline double sigm(double z) { return 1.0 / (1.0 + std::exp(-z)); }

}  // namespace

extern "C" {

// Camera centre p = -R^T t in float64.
void orc_camera_center(const orc_camera* c, double* out3) { center64(c, out3); }

// Unified camera for a stereo pair, Eq. 5-6 (Sec. 4, binocular de-redundancy):
//   d_u = mean(d_1, d_2) / |mean(d_1, d_2)|
//   p_u = mean(p_1, p_2) - d_u |p_1 - p_2| / (2 tan(theta/2)),
// with theta the horizontal field of view, so 2 tan(theta/2) = W / fx.
// The paper gives only the direction; the right/down axes are read as the
// mean down axis of the eyes orthogonalised against d_u.  Intrinsics are the
// left eye's.  Float64 arithmetic in a fixed order, rounded once to float32.
int orc_unified_camera(const orc_camera* L, const orc_camera* Rr, orc_camera* out) {
  if (!L || !Rr || !out) return -1;
  double p1[3], p2[3];
  center64(L, p1);
  center64(Rr, p2);
  double d[3], y[3], pm[3];
  for (int i = 0; i < 3; ++i) {
    d[i] = ((double)L->R[6 + i] + (double)Rr->R[6 + i]) * 0.5;
    y[i] = ((double)L->R[3 + i] + (double)Rr->R[3 + i]) * 0.5;
    pm[i] = (p1[i] + p2[i]) * 0.5;
  }
  double dn = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  double du[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
  double bx = p1[0] - p2[0], by = p1[1] - p2[1], bz = p1[2] - p2[2];
  double b = std::sqrt((bx * bx + by * by) + bz * bz);
  double back = (b * (double)L->fx) / (double)L->width;  // |p1-p2| / (2 tan(theta/2))
  double pu[3] = {pm[0] - du[0] * back, pm[1] - du[1] * back, pm[2] - du[2] * back};
  // x_u = normalize(y_ref x d_u); y_u = d_u x x_u
  double xr[3] = {y[1] * du[2] - y[2] * du[1], y[2] * du[0] - y[0] * du[2], y[0] * du[1] - y[1] * du[0]};
  double xn = std::sqrt((xr[0] * xr[0] + xr[1] * xr[1]) + xr[2] * xr[2]);
  double xu[3] = {xr[0] / xn, xr[1] / xn, xr[2] / xn};
  double yu[3] = {du[1] * xu[2] - du[2] * xu[1], du[2] * xu[0] - du[0] * xu[2], du[0] * xu[1] - du[1] * xu[0]};
  double Ru[9] = {xu[0], xu[1], xu[2], yu[0], yu[1], yu[2], du[0], du[1], du[2]};
  *out = *L;
  for (int i = 0; i < 9; ++i) out->R[i] = (float)Ru[i];
  for (int r = 0; r < 3; ++r) {
    double s = Ru[r * 3 + 0] * pu[0];
    s = s + Ru[r * 3 + 1] * pu[1];
    s = s + Ru[r * 3 + 2] * pu[2];
    out->t[r] = (float)(-s);
  }
  return 0;
}

// Anchor filtering (Sec. 3.2, Alg. 1 "anchors indexing and filtering"):
// frustum test with a 1.3 guard band and the distance LOD rule (an anchor of
// level l >= 1 is drawn iff its distance d to the camera satisfies
// d <= d_max 2^-l; level 0 is always drawn).  With Octree-GS level offsets
// (reading of Sec. 2's distance-chosen octree levels) level l >= 1 is drawn
// iff l <= log2(d_max / d) + Delta_a, i.e. d <= d_max 2^(Delta_a - l); the
// threshold is that radius taken once in float64 and rounded to float32,
//   thr = (float) ldexp(d_max * exp2(Delta_a), -l).
// Decision-pinned float32:
//   c = ((R0 x + R1 y) + R2 z) + t0   (and likewise for rows 1, 2)
//   c.z > znear  and |c.x| <= (1.3 tan_x) c.z  and |c.y| <= (1.3 tan_y) c.z,
//   tan_x = (0.5 W) / fx;   d^2 = (dx dx + dy dy) + dz dz <= (d_max 2^-l)^2.
// Writes the ascending ids of visible anchors; returns their count.
int64_t orc_cull(const orc_model* m, const orc_camera* c, uint32_t* ids, int64_t cap) {
  if (!m || !c) return -1;
  double p64[3];
  center64(c, p64);
  const float pcx = (float)p64[0], pcy = (float)p64[1], pcz = (float)p64[2];
  const float tanx = (0.5f * (float)c->width) / c->fx;
  const float tany = (0.5f * (float)c->height) / c->fy;
  const float gx = 1.3f * tanx, gy = 1.3f * tany;
  const float* R = c->R;
  std::vector<uint8_t> vis((size_t)m->n);
#pragma omp parallel for schedule(static)
  for (int64_t a = 0; a < m->n; ++a) {
    const float x = m->pos[3 * a], y = m->pos[3 * a + 1], z = m->pos[3 * a + 2];
    float X = R[0] * x; X = X + R[1] * y; X = X + R[2] * z; X = X + c->t[0];
    float Y = R[3] * x; Y = Y + R[4] * y; Y = Y + R[5] * z; Y = Y + c->t[1];
    float Z = R[6] * x; Z = Z + R[7] * y; Z = Z + R[8] * z; Z = Z + c->t[2];
    bool v = (Z > c->znear) && (std::fabs(X) <= gx * Z) && (std::fabs(Y) <= gy * Z);
    const int l = m->level[a];
    if (v && l >= 1) {
      float dx = x - pcx, dy = y - pcy, dz = z - pcz;
      float d2 = dx * dx;
      d2 = d2 + dy * dy;
      d2 = d2 + dz * dz;
      float thr;
      if (m->level_offset)
        thr = (float)std::ldexp((double)m->lod_dmax * std::exp2((double)m->level_offset[a]), -l);
      else
        thr = std::ldexp(m->lod_dmax, -l);
      v = d2 <= thr * thr;
    }
    vis[a] = v ? 1 : 0;
  }
  int64_t cnt = 0;
  for (int64_t a = 0; a < m->n; ++a)
    if (vis[a]) {
      if (ids && cnt < cap) ids[cnt] = (uint32_t)a;
      ++cnt;
    }
  return cnt;
}

// Octree-GS level fade (reading: a level is switched on gradually).  For a
// visible anchor of level l >= 1, u = log2(r_a / d) is how many levels it
// lies inside its switching distance; its Gaussians' opacities are scaled by
// w = clamp(u / beta, 0, 1); level 0 (and beta = 0) give w = 1.  r_a is the
// culling radius and d^2 the culling test's pinned float32 squared distance
// (so u >= 0 for every kept anchor); u itself is float64:
//   u = log1p((r_a^2 - d^2) / d^2) / (2 ln 2).
int orc_lod_weight(const orc_model* m, const orc_camera* c, const uint32_t* ids, int64_t n, double beta,
                   double* w) {
  if (!m || !c || (n > 0 && (!ids || !w))) return -1;
  double p64[3];
  center64(c, p64);
  const float pcx = (float)p64[0], pcy = (float)p64[1], pcz = (float)p64[2];
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t a = ids[i];
    const int l = m->level[a];
    if (!(beta > 0.0) || l == 0) {
      w[i] = 1.0;
      continue;
    }
    const double delta = m->level_offset ? (double)m->level_offset[a] : 0.0;
    const float r = (float)std::ldexp((double)m->lod_dmax * std::exp2(delta), -l);
    const float x = m->pos[3 * (size_t)a], y = m->pos[3 * (size_t)a + 1], z = m->pos[3 * (size_t)a + 2];
    float dx = x - pcx, dy = y - pcy, dz = z - pcz;
    float d2 = dx * dx;
    d2 = d2 + dy * dy;
    d2 = d2 + dz * dz;
    const double r2 = (double)r * (double)r;  // exact
    const double u = std::log1p((r2 - (double)d2) / (double)d2) / (2.0 * std::log(2.0));
    w[i] = std::min(1.0, std::max(0.0, u / beta));
  }
  return 0;
}

// Derivation, Eq. 3 (Sec. 3.1): for each anchor a,
//   d = (x_a - p) / |x_a - p|, x = [f_a ; d]  (35 values),
//   per head h in {opacity, colour, covariance}:
//     z_h = W2_h^T ReLU(W1_h^T x + b1_h) + b2_h,
//   and for Gaussian j < k:
//     alpha_j = tanh(z_op[j])             kept iff alpha_j > 0  (mask, Sec. 6)
//     c_j     = sigmoid(z_col[3j..3j+2])
//     s_j     = s_a * sigmoid(z_cov[7j..7j+2])
//     q_j     = z_cov[7j+3..7j+6] / |.|    (w, x, y, z); identity if |.| < 1e-12
// attrs: [n][k][11] = alpha, c(3), s(3), q(4); kept: [n][k].
// With q->mode != 0 the inputs, weights and hidden activations are rounded as
// the precision form does (the sums stay float64): mode 1 all to bf16; mode 2
// (FP8-E4M3, per-tensor power-of-two scales) the inputs to one E4M3 term and
// the weights and hidden activations to two-term E4M3 expansions, the second
// layer summing h_hi W_hi + h_lo W_hi + h_hi W_lo (no h_lo W_lo term).
int orc_derive(const orc_model* m, const double* view_pos, const uint32_t* ids, int64_t n,
               const orc_quant* qz, double* attrs, uint8_t* kept, double* raw_out) {
  if (!m || !ids || !attrs) return -1;
  const int k = m->k;
  const int outd[3] = {k, 3 * k, 7 * k};
  const int mode = qz ? qz->mode : 0;
  // pre-round the weights once (FP8: W2q holds the leading term of each
  // W2 weight, W2r the second; W1q the two-term sum)
  std::vector<double> W1q[3], W2q[3], W2r[3];
  for (int h = 0; h < 3; ++h) {
    W1q[h].resize(IN * HID);
    W2q[h].resize((size_t)HID * outd[h]);
    W2r[h].assign((size_t)HID * outd[h], 0.0);
    for (int i = 0; i < IN * HID; ++i) {
      float w = m->W1[h][i];
      if (mode == 1) W1q[h][i] = round_bf16(w);
      else if (mode == 2) W1q[h][i] = e4m3_two_term(w, qz->s_w1[h], nullptr);
      else W1q[h][i] = w;
    }
    for (int i = 0; i < HID * outd[h]; ++i) {
      float w = m->W2[h][i];
      if (mode == 1) W2q[h][i] = round_bf16(w);
      else if (mode == 2) {
        double hi;
        const double all = e4m3_two_term(w, qz->s_w2[h], &hi);
        W2q[h][i] = hi;
        W2r[h][i] = all - hi;
      } else W2q[h][i] = w;
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t a = ids[i];
    double v[3];
    for (int c = 0; c < 3; ++c) v[c] = (double)m->pos[3 * (size_t)a + c] - view_pos[c];
    double vn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double x[IN];
    for (int c = 0; c < FDIM; ++c) x[c] = m->feat[(size_t)a * FDIM + c];
    for (int c = 0; c < 3; ++c) x[FDIM + c] = v[c] / vn;
    if (mode == 1) {
      for (int c = 0; c < IN; ++c) x[c] = round_bf16((float)x[c]);
    } else if (mode == 2) {
      for (int c = 0; c < IN; ++c) x[c] = round_e4m3(x[c] / qz->s_x) * qz->s_x;
    }
    double z[3][7 * 16];
    for (int h = 0; h < 3; ++h) {
      double hid[HID], hlo[HID];
      for (int o = 0; o < HID; ++o) {
        double s = 0.0;
        for (int c = 0; c < IN; ++c) s += x[c] * W1q[h][c * HID + o];
        s += (double)m->b1[h][o];
        s = s > 0.0 ? s : 0.0;
        hlo[o] = 0.0;
        if (mode == 1) s = round_bf16((float)s);
        else if (mode == 2) {
          double hi;
          const double all = e4m3_two_term(s, qz->s_h[h], &hi);
          hlo[o] = all - hi;
          s = hi;
        }
        hid[o] = s;
      }
      // FP8: (h_hi + h_lo)(W_hi + W_lo) without the h_lo W_lo term
      for (int o = 0; o < outd[h]; ++o) {
        double s = 0.0;
        for (int c = 0; c < HID; ++c) {
          const size_t wi = (size_t)c * outd[h] + o;
          s += hid[c] * W2q[h][wi];
          if (mode == 2) s += hlo[c] * W2q[h][wi] + hid[c] * W2r[h][wi];
        }
        z[h][o] = s + (double)m->b2[h][o];
      }
    }
    if (raw_out) {
      double* r = raw_out + (size_t)i * 11 * k;
      int p = 0;
      for (int h = 0; h < 3; ++h)
        for (int o = 0; o < outd[h]; ++o) r[p++] = z[h][o];
    }
    const double sa = m->scale[a];
    for (int j = 0; j < k; ++j) {
      double* at = attrs + ((size_t)i * k + j) * 11;
      double al = std::tanh(z[0][j]);
      at[0] = al;
      if (kept) kept[(size_t)i * k + j] = al > 0.0 ? 1 : 0;
      for (int c = 0; c < 3; ++c) at[1 + c] = sigm(z[1][3 * j + c]);
      for (int c = 0; c < 3; ++c) at[4 + c] = sa * sigm(z[2][7 * j + c]);
      double q[4] = {z[2][7 * j + 3], z[2][7 * j + 4], z[2][7 * j + 5], z[2][7 * j + 6]};
      double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      if (qn < 1e-12) {
        at[7] = 1.0; at[8] = 0.0; at[9] = 0.0; at[10] = 0.0;
      } else {
        for (int c = 0; c < 4; ++c) at[7 + c] = q[c] / qn;
      }
    }
  }
  return 0;
}

// Rotation matrix of a unit quaternion (w, x, y, z).
void orc_quat_to_rot(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z); R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y); R[7] = 2.0 * (y * z + w * x); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Projection of one 3D Gaussian (Eq. 1-2 and the EWA splatting step of
// Sec. 3.1):
//   Sigma = R(q) diag(s^2) R(q)^T                                   (Eq. 2)
//   t = W mu + t_cam;  J = [[fx/tz, 0, -fx tx'/tz^2], [0, fy/tz, -fy ty'/tz^2]]
//   with tx' = clamp(tx/tz, +-1.3 tan_x) tz (and likewise ty');
//   Sigma' = J W Sigma W^T J^T + 0.3 I;   mean = (fx tx/tz + cx, fy ty/tz + cy).
// out[0..10] = mean x, mean y, Sigma'xx, Sigma'xy, Sigma'yy, conic A, B, C,
// depth tz, det, valid.  The near-plane drop is decided by the caller on the
// pinned float32 depth.
void orc_project_gaussian(const orc_camera* c, const double* mu, const double* s, const double* q,
                          double* out) {
  const float* Rc = c->R;
  double W[9];
  for (int i = 0; i < 9; ++i) W[i] = Rc[i];
  double t[3];
  for (int r = 0; r < 3; ++r) t[r] = W[3 * r] * mu[0] + W[3 * r + 1] * mu[1] + W[3 * r + 2] * mu[2] + (double)c->t[r];
  const double fx = c->fx, fy = c->fy;
  const double tanx = (0.5 * c->width) / fx, tany = (0.5 * c->height) / fy;
  const double limx = 1.3 * tanx, limy = 1.3 * tany;
  const double tz = t[2];
  double txz = t[0] / tz, tyz = t[1] / tz;
  txz = std::min(limx, std::max(-limx, txz));
  tyz = std::min(limy, std::max(-limy, tyz));
  const double txc = txz * tz, tyc = tyz * tz;
  double J[6] = {fx / tz, 0.0, -fx * txc / (tz * tz), 0.0, fy / tz, -fy * tyc / (tz * tz)};
  double Rq[9];
  orc_quat_to_rot(q, Rq);
  double S[9];  // Sigma = Rq diag(s^2) Rq^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += Rq[3 * i + l] * s[l] * s[l] * Rq[3 * j + l];
      S[3 * i + j] = acc;
    }
  double T[6];  // T = J W  (2x3)
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += J[3 * i + l] * W[3 * l + j];
      T[3 * i + j] = acc;
    }
  double M[6];  // M = T S (2x3)
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += T[3 * i + l] * S[3 * l + j];
      M[3 * i + j] = acc;
    }
  double cxx = 0, cxy = 0, cyy = 0;
  for (int l = 0; l < 3; ++l) {
    cxx += M[l] * T[l];
    cxy += M[l] * T[3 + l];
    cyy += M[3 + l] * T[3 + l];
  }
  cxx += 0.3;
  cyy += 0.3;
  const double det = cxx * cyy - cxy * cxy;
  out[0] = fx * t[0] / tz + (double)c->cx;
  out[1] = fy * t[1] / tz + (double)c->cy;
  out[2] = cxx; out[3] = cxy; out[4] = cyy;
  out[5] = cyy / det; out[6] = -cxy / det; out[7] = cxx / det;
  out[8] = tz;
  out[9] = det;
  out[10] = (det > 0.0) ? 1.0 : 0.0;
}

// Pinned float32 depth used to order Gaussians (an integer decision):
//   mu32 = x_a + o  (float32 adds), tz32 = ((W6 mu_x + W7 mu_y) + W8 mu_z) + t2.
float orc_depth32(const orc_camera* c, const float* xa, const float* o) {
  const float mx = xa[0] + o[0], my = xa[1] + o[1], mz = xa[2] + o[2];
  const float* R = c->R;
  float z = R[6] * mx;
  z = z + R[7] * my;
  z = z + R[8] * mz;
  z = z + c->t[2];
  return z;
}

// Records of one view from derived attributes.  Record r = i*k + j for
// visible index i and Gaussian j (ascending global id a*k + j).  Per record
// (stride ORC_REC = 16 doubles): valid, mean x, mean y, conic A, B, C,
// opacity, colour r, g, b, depth (fp64), tau = 2 ln(255 o), Sigma'xx, xy, yy,
// e_mean.  depth32 is the pinned ordering depth.  e_mean (pixels) is the
// distance a float32 evaluation of the projection can move the 2D mean:
// the camera-relative position, the rotation sums and the perspective
// divide each carry an error of a few float32 ulps of the quantities they
// combine, which at the image reaches f (1 + |x'| + |y'|)(1 + max(|x'|, |y'|))
// ulps of a unit (x' = (m_x - c_x) / f_x, y' = (m_y - c_y) / f_y: the
// tangent offsets), independent of depth; the term takes 4 such ulps
// (2^-22) of that plus of max(|m_x|, |m_y|), per axis its larger value.  A record is valid iff the
// Gaussian is kept (alpha > 0), its pinned depth is > znear and det > 0.
int orc_project_records(const orc_model* m, const orc_camera* c, const uint32_t* ids, int64_t n,
                        const double* attrs, const uint8_t* kept, double* rec, float* depth32) {
  if (!m || !c || !ids || !attrs || !rec || !depth32) return -1;
  const int k = m->k;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t a = ids[i];
    const float* xa = m->pos + 3 * (size_t)a;
    for (int j = 0; j < k; ++j) {
      const size_t r = (size_t)i * k + j;
      const double* at = attrs + r * 11;
      const float* o = m->offs + ((size_t)a * k + j) * 3;
      double* out = rec + r * 16;
      std::memset(out, 0, 16 * sizeof(double));
      float d32 = orc_depth32(c, xa, o);
      depth32[r] = d32;
      const bool keep = kept ? kept[r] != 0 : at[0] > 0.0;
      if (!keep || !(d32 > c->znear)) continue;
      double mu[3] = {(double)xa[0] + (double)o[0], (double)xa[1] + (double)o[1], (double)xa[2] + (double)o[2]};
      double pr[11];
      orc_project_gaussian(c, mu, at + 4, at + 7, pr);
      if (pr[10] == 0.0) continue;
      out[0] = 1.0;
      out[1] = pr[0]; out[2] = pr[1];
      out[3] = pr[5]; out[4] = pr[6]; out[5] = pr[7];
      out[6] = at[0];
      out[7] = at[1]; out[8] = at[2]; out[9] = at[3];
      out[10] = pr[8];
      out[11] = 2.0 * std::log(255.0 * at[0]);
      out[12] = pr[2]; out[13] = pr[3]; out[14] = pr[4];
      const double ux = std::fabs(pr[0] - (double)c->cx) / (double)c->fx;
      const double uy = std::fabs(pr[1] - (double)c->cy) / (double)c->fy;
      const double sp = (1.0 + ux + uy) * (1.0 + std::max(ux, uy));
      const double mm = std::max(std::fabs(pr[0]), std::fabs(pr[1]));
      out[15] = std::ldexp(std::max((double)c->fx, (double)c->fy) * sp + mm, -22);
    }
  }
  return 0;
}

}  // extern "C"

namespace {

// Tiles covered by the ellipse q(D) = A Dx^2 + 2 B Dx Dy + C Dy^2 <= tau, where
// a tile is covered iff the hull of its pixel centres meets the ellipse
// (Sec. 6: opacity-aware extent + exact tile coverage).  Per tile row the
// ellipse restricted to the row's band of pixel-centre y is convex, so its
// x-range is [x_min, x_max] with the extremes found in closed form:
//   the point of largest x lies at Dy* = -B sqrt(tau / (C det)), the point of
//   smallest x at -Dy*; clamped into the band they give
//   x_max = (-B y + sqrt(A tau - det y^2)) / A,  x_min = (-B y - sqrt(...)) / A.
template <typename F, typename Emit>
void cover_tiles(F mx, F my, F A, F B, F C, F tau, int W, int H, int TW, int TH, Emit emit) {
  const F det = A * C - B * B;
  if (!(tau > F(0)) || !(det > F(0)) || !(A > F(0)) || !(C > F(0))) return;
  const int ntx = (W + TW - 1) / TW, nty = (H + TH - 1) / TH;
  const F ey = std::sqrt((tau * A) / det);
  const F ys = (-B) * std::sqrt(tau / (C * det));
  const F fTW = (F)TW, fTH = (F)TH;
  F fy0 = std::ceil((((my - ey) - (fTH - F(0.5))) / fTH));
  F fy1 = std::floor(((my + ey) - F(0.5)) / fTH);
  fy0 = std::fmin(std::fmax(fy0, F(0)), (F)nty);
  fy1 = std::fmin(std::fmax(fy1, F(-1)), (F)(nty - 1));
  const int ty0 = (int)fy0, ty1 = (int)fy1;
  for (int ty = ty0; ty <= ty1; ++ty) {
    F b0 = ((F)(ty * TH) + F(0.5)) - my;
    F b1 = ((F)(ty * TH + TH) - F(0.5)) - my;
    b0 = std::fmax(b0, -ey);
    b1 = std::fmin(b1, ey);
    if (b0 > b1) continue;
    const F yr = std::fmin(std::fmax(ys, b0), b1);
    const F yl = std::fmin(std::fmax(-ys, b0), b1);
    const F dr = (A * tau) - (det * (yr * yr));
    const F dl = (A * tau) - (det * (yl * yl));
    const F xr = (((-B) * yr) + std::sqrt(std::fmax(dr, F(0)))) / A;
    const F xl = (((-B) * yl) - std::sqrt(std::fmax(dl, F(0)))) / A;
    F fx0 = std::ceil(((mx + xl) - (fTW - F(0.5))) / fTW);
    F fx1 = std::floor(((mx + xr) - F(0.5)) / fTW);
    fx0 = std::fmin(std::fmax(fx0, F(0)), (F)ntx);
    fx1 = std::fmin(std::fmax(fx1, F(-1)), (F)(ntx - 1));
    const int tx0 = (int)fx0, tx1 = (int)fx1;
    for (int tx = tx0; tx <= tx1; ++tx) emit(ty * ntx + tx);
  }
}

struct Pair {
  uint32_t tile;
  uint32_t dbits;
  int64_t gid;
  int64_t idx;
};

inline uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

}  // namespace

extern "C" {

// Exact tile list of one ellipse, float64 (oracle tiling) - for tests.
int64_t orc_cover_tiles64(double mx, double my, double A, double B, double C, double tau, int W, int H,
                          int TW, int TH, int32_t* out, int64_t cap) {
  int64_t n = 0;
  cover_tiles<double>(mx, my, A, B, C, tau, W, H, TW, TH, [&](int t) {
    if (out && n < cap) out[n] = t;
    ++n;
  });
  return n;
}

// Stage-isolated float32 key generation: the same coverage definition
// evaluated in float32 with a fixed operation order, applied to float32
// records produced elsewhere.  Emits, in record order, key = view * n_tiles +
// tile and value = record index.  Returns the number of pairs.
int64_t orc_keygen_f32(int64_t n, const float* mx, const float* my, const float* A, const float* B,
                       const float* C, const float* tau, const int32_t* view, const uint8_t* valid,
                       int W, int H, int TW, int TH, uint32_t* counts, uint32_t* keys, uint32_t* vals,
                       int64_t cap) {
  const int ntiles = ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
  int64_t p = 0;
  for (int64_t r = 0; r < n; ++r) {
    uint32_t cnt = 0;
    if (!valid || valid[r]) {
      const uint32_t base = (uint32_t)view[r] * (uint32_t)ntiles;
      cover_tiles<float>(mx[r], my[r], A[r], B[r], C[r], tau[r], W, H, TW, TH, [&](int t) {
        if (keys && p < cap) {
          keys[p] = base + (uint32_t)t;
          vals[p] = (uint32_t)r;
        }
        ++p;
        ++cnt;
      });
    }
    if (counts) counts[r] = cnt;
  }
  return p;
}

// Front-to-back alpha blending (Sec. 3.1), per pixel, over the Gaussians in
// (pinned depth ascending, global id ascending) order:
//   D = (px + 0.5, py + 0.5) - mean;  q = A Dx^2 + 2 B Dx Dy + C Dy^2
//   alpha = min(0.99, o exp(-q/2)); skip if alpha < 1/255;
//   stop before adding a Gaussian if T (1 - alpha) < 1e-4;
//   C += c alpha T;  T *= (1 - alpha);   output C + T bg.
// mode 0 = brute force: every Gaussian at every pixel.  mode 1 = tiled: each
// pixel only visits the Gaussians whose exact tile coverage (float64, with
// tau enlarged by 2^-7 relative + 2^-7 so the tile set is a strict superset
// of the alpha >= 1/255 region and also holds the Gaussians just outside it,
// whose margins matter) contains its tile; the images are identical.
// rec: [n][16] as written by orc_project_records; gid: global Gaussian ids.
// Pixel list px/py (npix >= 0) or all pixels (npix < 0, row-major output).
// margin: per pixel, the smallest |ln(alpha_raw * 255)| and |ln(T(1-alpha) 1e4)|
// over the Gaussians the pixel evaluated (how close a threshold decision was).
// walk (optional): per pixel, how many Gaussians of its list it evaluated -
// all of them, or up to and including the one at which it stops.
int orc_render(const double* rec, const float* depth32, const int64_t* gid, int64_t n, int W, int H,
               int mode, int TW, int TH, int64_t npix, const int32_t* px, const int32_t* py,
               const double* bg, double* out_rgb, double* out_T, double* out_margin,
               int32_t* out_ncontrib, int32_t* out_walk) {
  if (!rec || !depth32 || !gid || !out_rgb) return -1;
  // order of all valid records
  std::vector<int64_t> order;
  order.reserve((size_t)n);
  for (int64_t r = 0; r < n; ++r)
    if (rec[r * 16] != 0.0) order.push_back(r);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const uint32_t da = fbits(depth32[a]), db = fbits(depth32[b]);
    if (da != db) return da < db;
    return gid[a] < gid[b];
  });
  const bool all = npix < 0;
  const int64_t NP = all ? (int64_t)W * H : npix;
  const int ntx = (W + TW - 1) / TW, nty = (H + TH - 1) / TH;
  std::vector<int64_t> tstart, tlist;
  if (mode == 1) {
    // keys (tile, depth bits, gid) for every covered pair of a needed tile
    std::vector<uint8_t> need((size_t)ntx * nty, all ? 1 : 0);
    if (!all)
      for (int64_t i = 0; i < NP; ++i) need[(size_t)(py[i] / TH) * ntx + px[i] / TW] = 1;
    std::vector<Pair> pairs;
    for (int64_t r : order) {
      const double* g = rec + r * 16;
      const double tau = g[11] * (1.0 + std::ldexp(1.0, -7)) + std::ldexp(1.0, -7);
      cover_tiles<double>(g[1], g[2], g[3], g[4], g[5], tau, W, H, TW, TH, [&](int t) {
        if (need[(size_t)t]) pairs.push_back(Pair{(uint32_t)t, fbits(depth32[r]), gid[r], r});
      });
    }
    std::sort(pairs.begin(), pairs.end(), [](const Pair& a, const Pair& b) {
      if (a.tile != b.tile) return a.tile < b.tile;
      if (a.dbits != b.dbits) return a.dbits < b.dbits;
      return a.gid < b.gid;
    });
    tstart.assign((size_t)ntx * nty + 1, 0);
    for (const Pair& p : pairs) tstart[p.tile + 1]++;
    for (size_t t = 0; t < (size_t)ntx * nty; ++t) tstart[t + 1] += tstart[t];
    tlist.resize(pairs.size());
    for (size_t i = 0; i < pairs.size(); ++i) tlist[i] = pairs[i].idx;
  }
  const double bgv[3] = {bg ? bg[0] : 0.0, bg ? bg[1] : 0.0, bg ? bg[2] : 0.0};
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < NP; ++i) {
    const int x = all ? (int)(i % W) : px[i];
    const int y = all ? (int)(i / W) : py[i];
    const double X = x + 0.5, Y = y + 0.5;
    double T = 1.0, Cc[3] = {0, 0, 0}, mg = 1e300;
    int nc = 0;
    const int64_t* lst;
    int64_t len;
    if (mode == 1) {
      const size_t t = (size_t)(y / TH) * ntx + x / TW;
      lst = tlist.data() + tstart[t];
      len = tstart[t + 1] - tstart[t];
    } else {
      lst = order.data();
      len = (int64_t)order.size();
    }
    int64_t walk = len;
    for (int64_t u = 0; u < len; ++u) {
      const double* g = rec + lst[u] * 16;
      const double dx = X - g[1], dy = Y - g[2];
      const double q = g[3] * dx * dx + 2.0 * g[4] * dx * dy + g[5] * dy * dy;
      const double araw = g[6] * std::exp(-0.5 * q);
      const double al = std::min(0.99, araw);
      // distance of the 1/255 decision from its threshold in log-opacity,
      // less what a float32 projection's error in the mean can move it: an
      // error e in the mean shifts q/2 by up to |grad_mean(q/2)|_1 e, with e
      // the record's e_mean
      const double grad = std::fabs(g[3] * dx + g[4] * dy) + std::fabs(g[4] * dx + g[5] * dy);
      const double ma = std::fabs(std::log(araw * 255.0)) - grad * g[15];
      if (ma < mg) mg = ma;
      if (al < 1.0 / 255.0) continue;
      const double tt = T * (1.0 - al);
      const double ms = std::fabs(std::log(tt * 1e4));
      if (ms < mg) mg = ms;
      if (tt < 1e-4) {
        walk = u + 1;
        break;
      }
      for (int c = 0; c < 3; ++c) Cc[c] += g[7 + c] * al * T;
      T = tt;
      ++nc;
    }
    for (int c = 0; c < 3; ++c) out_rgb[i * 3 + c] = Cc[c] + T * bgv[c];
    if (out_T) out_T[i] = T;
    if (out_margin) out_margin[i] = mg;
    if (out_ncontrib) out_ncontrib[i] = nc;
    if (out_walk) out_walk[i] = (int32_t)walk;
  }
  return 0;
}

// Blend trace of one pixel over an explicit ordered list of (alpha_raw, colour)
// - the blending rule alone, for the invariant tests.  Writes, per visited
// entry, [alpha used (or -1 if skipped), T before, weight]; returns the
// number of entries visited (the stop entry included).
int64_t orc_blend_trace(const double* araw, const double* col, int64_t n, double* trace, double* out_rgbT) {
  double T = 1.0, C[3] = {0, 0, 0};
  int64_t u = 0;
  for (; u < n; ++u) {
    const double al = std::min(0.99, araw[u]);
    if (al < 1.0 / 255.0) {
      trace[3 * u] = -1.0; trace[3 * u + 1] = T; trace[3 * u + 2] = 0.0;
      continue;
    }
    const double tt = T * (1.0 - al);
    if (tt < 1e-4) {
      trace[3 * u] = al; trace[3 * u + 1] = T; trace[3 * u + 2] = 0.0;
      ++u;
      break;
    }
    const double w = al * T;
    for (int c = 0; c < 3; ++c) C[c] += col[3 * u + c] * w;
    trace[3 * u] = al; trace[3 * u + 1] = T; trace[3 * u + 2] = w;
    T = tt;
  }
  out_rgbT[0] = C[0]; out_rgbT[1] = C[1]; out_rgbT[2] = C[2]; out_rgbT[3] = T;
  return u;
}

// Format conversions used by the precision forms (exposed for their pins).
float orc_round_bf16(float x) { return round_bf16(x); }
double orc_round_e4m3(double x) { return round_e4m3(x); }

double orc_e4m3_two_term(double v, double s, double* hi) { return e4m3_two_term(v, s, hi); }

// Threads of the parallel loops (timing the oracle at 1 thread and at all
// cores); the arithmetic and its order per pixel / anchor do not depend on it.
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"

// FP64 oracle of the radiance-cache MLP (test infrastructure only).
//
// Network (radiance cache added around the path tracer; the paper itself only
// names caches as an open direction, Sec. 3.2): a 64-dimensional encoding of
// (position, direction, normal, roughness), five 64x64 ReLU layers and a 64x3
// linear head, no biases (three constant-one inputs play that role).  The
// kernels keep weights and inter-layer activations in BF16 and accumulate in
// FP32; this oracle accumulates in FP64 and rounds to BF16 at the same points
// (encoding, every ReLU output, every weight), so the two differ only by
// accumulation rounding and by rare BF16 rounding-boundary flips.
// Loss: relative L2 of Mueller et al. 2021 (Real-time Neural Radiance
// Caching): mean over the batch of sum_c (y_c - t_c)^2 / (sg(y_c)^2 + 0.01).
// Optimiser: Adam (Kingma & Ba 2015).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int kW = 64;      // width
constexpr int kHidden = 5;  // hidden 64x64 layers (the first consumes the encoding)
constexpr int kOut = 3;
constexpr int kParams = kHidden * kW * kW + kOut * kW;
constexpr double kPi = 3.14159265358979323846;

// BF16 rounding can be switched off so that finite differences can check the
// backward pass of the plain FP64 network.
int g_round = 1;

// Round to the nearest BF16 value (ties to even), via FP32.
double bf16(double x) {
  if (!g_round) return x;
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;  // inf / nan unchanged
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// Encoding of one raw record (p[3], w[3], n[3], alpha) -> 64 values (before BF16 rounding).
// p is normalised to the cache's box; frequencies 2^k pi, k < 6 for p, k < 2 for w, n
// (which are mapped from [-1,1] to [0,1] first).
void encode(const double* raw, const double* lo, const double* hi, double* e) {
  int j = 0;
  for (int a = 0; a < 3; ++a) {
    double x = (raw[a] - lo[a]) / (hi[a] - lo[a]);
    for (int k = 0; k < 6; ++k) {
      double ang = std::ldexp(kPi, k) * x;
      e[j++] = std::sin(ang);
      e[j++] = std::cos(ang);
    }
  }
  for (int v = 0; v < 2; ++v) {
    for (int a = 0; a < 3; ++a) {
      double x = 0.5 * (raw[3 + 3 * v + a] + 1.0);
      for (int k = 0; k < 2; ++k) {
        double ang = std::ldexp(kPi, k) * x;
        e[j++] = std::sin(ang);
        e[j++] = std::cos(ang);
      }
    }
  }
  e[j++] = raw[9];
  e[j++] = 1.0;
  e[j++] = 1.0;
  e[j++] = 1.0;
}

struct Acts {
  double x[kHidden + 1][kW];  // inputs of each layer (x[0] = encoding), BF16-rounded
  double y[kOut];
};

void forward(const double* W, const double* enc, Acts& a) {
  for (int i = 0; i < kW; ++i) a.x[0][i] = bf16(enc[i]);
  for (int l = 0; l < kHidden; ++l) {
    const double* Wl = W + (size_t)l * kW * kW;
    for (int o = 0; o < kW; ++o) {
      double s = 0.0;
      for (int i = 0; i < kW; ++i) s += bf16(Wl[o * kW + i]) * a.x[l][i];
      a.x[l + 1][o] = bf16(s > 0.0 ? s : 0.0);
    }
  }
  const double* Wo = W + (size_t)kHidden * kW * kW;
  for (int o = 0; o < kOut; ++o) {
    double s = 0.0;
    for (int i = 0; i < kW; ++i) s += bf16(Wo[o * kW + i]) * a.x[kHidden][i];
    a.y[o] = s;
  }
}

}  // namespace

extern "C" {

int oracle_mlp_n_params() { return kParams; }

void oracle_mlp_set_rounding(int on) { g_round = on; }

// raw: [n][10]; box: lo[3], hi[3]; enc_out: [n][64] (BF16-rounded values)
void oracle_nrc_encode(int n, const double* raw, const double* box, double* enc_out) {
  const double* lo = box;
  const double* hi = box + 3;
  for (int r = 0; r < n; ++r) {
    double e[kW];
    encode(raw + 10 * (size_t)r, lo, hi, e);
    for (int i = 0; i < kW; ++i) enc_out[(size_t)r * kW + i] = bf16(e[i]);
  }
}

// W: [kParams] (rounded to BF16 inside); enc: [n][64]; out: [n][3]
void oracle_mlp_forward(const double* W, int n, const double* enc, double* out) {
  for (int r = 0; r < n; ++r) {
    Acts a;
    forward(W, enc + (size_t)r * kW, a);
    for (int o = 0; o < kOut; ++o) out[(size_t)r * kOut + o] = a.y[o];
  }
}

// Relative-L2 loss over a batch and its gradient with respect to the weights
// (grad: [kParams], gradients w.r.t. the BF16-rounded weights).  Returns the loss.
double oracle_mlp_loss_grad(const double* W, int n, const double* enc, const double* target, double* grad,
                            double* out) {
  std::memset(grad, 0, sizeof(double) * kParams);
  double loss = 0.0;
  for (int r = 0; r < n; ++r) {
    Acts a;
    forward(W, enc + (size_t)r * kW, a);
    double dy[kOut];
    for (int o = 0; o < kOut; ++o) {
      double y = a.y[o], t = target[(size_t)r * kOut + o];
      double den = y * y + 0.01;
      loss += (y - t) * (y - t) / den / n;
      dy[o] = 2.0 * (y - t) / den / n;
      if (out) out[(size_t)r * kOut + o] = y;
    }
    // head
    double* Go = grad + (size_t)kHidden * kW * kW;
    const double* Wo = W + (size_t)kHidden * kW * kW;
    double dx[kW];
    for (int i = 0; i < kW; ++i) {
      double s = 0.0;
      for (int o = 0; o < kOut; ++o) {
        Go[o * kW + i] += dy[o] * a.x[kHidden][i];
        s += bf16(Wo[o * kW + i]) * dy[o];
      }
      dx[i] = s;
    }
    for (int l = kHidden - 1; l >= 0; --l) {
      // through the ReLU that produced x[l+1]
      double dz[kW];
      for (int o = 0; o < kW; ++o) dz[o] = a.x[l + 1][o] > 0.0 ? dx[o] : 0.0;
      double* Gl = grad + (size_t)l * kW * kW;
      const double* Wl = W + (size_t)l * kW * kW;
      double nx[kW];
      for (int i = 0; i < kW; ++i) {
        double s = 0.0;
        for (int o = 0; o < kW; ++o) {
          Gl[o * kW + i] += dz[o] * a.x[l][i];
          s += bf16(Wl[o * kW + i]) * dz[o];
        }
        nx[i] = s;
      }
      std::memcpy(dx, nx, sizeof dx);
    }
  }
  return loss;
}

// One Adam step on FP64 master weights; m, v: state; t: step number (1-based).
void oracle_mlp_adam(double* W, const double* grad, double* m, double* v, int t, double lr, double b1, double b2,
                     double eps, int n) {
  double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (int i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    W[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

}  // extern "C"

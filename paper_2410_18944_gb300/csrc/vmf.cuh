// von Mises-Fisher mixtures on S^{d-1} (Sec. 3.3, Eq. vmm) in FP32, the
// normalisation map of Tab. reg_map, and the two samplers the paper names:
// Best & Fisher (1979) rejection for d = 2 and the stable inverse-CDF form
// of Tokuyoshi (2025) for d = 3 (cos theta = 1 + log1p(xi expm1(-2k)) / k),
// with the orthonormal frame of Duff et al. (2017).
//
// Densities in exponentially scaled form:
//   d = 2: v = exp(-k |mu - nu|^2 / 2) / (2 pi I0e(k))
//   d = 3: v = k exp(-k |mu - nu|^2 / 2) / (2 pi (-expm1(-2k)))
// (k (mu.nu - 1) = -k |mu - nu|^2 / 2 for unit vectors, which avoids the
// cancellation of mu.nu - 1 near the mode).  I0e, I1e use the polynomial
// approximations 9.8.1-9.8.4 of Abramowitz & Stegun (1964), relative error
// below 2.2e-7.
#pragma once
#include "common.cuh"

namespace wost {

constexpr int kMaxKTheta = 8;

__device__ __forceinline__ float i0e_as(float x) {
    if (x <= 3.75f) {
        float t = x * (1.f / 3.75f);
        t *= t;
        float p = 1.f + t * (3.5156229f + t * (3.0899424f + t * (1.2067492f + t * (0.2659732f + t * (0.0360768f + t * 0.0045813f)))));
        return p * __expf(-x);
    }
    float t = 3.75f / x;
    float p = 0.39894228f + t * (0.01328592f + t * (0.00225319f + t * (-0.00157565f + t * (0.00916281f +
              t * (-0.02057706f + t * (0.02635537f + t * (-0.01647633f + t * 0.00392377f)))))));
    return p * rsqrtf(x);
}

__device__ __forceinline__ float i1e_as(float x) {
    if (x <= 3.75f) {
        float t = x * (1.f / 3.75f);
        t *= t;
        float p = 0.5f + t * (0.87890594f + t * (0.51498869f + t * (0.15084934f + t * (0.02658733f + t * (0.00301532f + t * 0.00032411f)))));
        return x * p * __expf(-x);
    }
    float t = 3.75f / x;
    float p = 0.39894228f + t * (-0.03988024f + t * (-0.00362018f + t * (0.00163801f + t * (-0.01031555f +
              t * (0.02282967f + t * (-0.02895312f + t * (0.01787654f - t * 0.00420059f)))))));
    return p * rsqrtf(x);
}

// log of the normalising factor: v = exp(-k |mu - nu|^2 / 2 + lognorm(k))
template <int D>
__device__ __forceinline__ float vmf_lognorm(float k) {
    if (D == 2) return -__logf(2.f * WOST_PI * i0e_as(k));
    return __logf(k / (2.f * WOST_PI * -expm1f(-2.f * k)));
}

// mean resultant length A_d(k) = E[mu . nu] = d log(normaliser) / dk + 1
template <int D>
__device__ __forceinline__ float vmf_mean_cos(float k) {
    if (D == 2) return i1e_as(k) / i0e_as(k);
    if (k < 0.02f) return k * (1.f / 3.f) - k * k * k * (1.f / 45.f);
    return 1.f / tanhf(k) - 1.f / k;
}

template <int D>
__device__ __forceinline__ float half_dist2(const float *mu, const float *nu) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) { float d = mu[i] - nu[i]; s += d * d; }
    return 0.5f * s;
}

// Normalised mixture parameters of one position (Tab. reg_map), room for
// KC lobes.
template <int D, int KC = kMaxKTheta>
struct Mixture {
    float mu[KC * D];
    float kappa[KC];
    float lam[KC];
    float lognorm[KC];
    float c;
};

// raw layout: mu'_i (K x d), kappa'_i (K), lambda'_i (K), c'
template <int D, int K, int KC>
__device__ __forceinline__ void theta_map(const float *raw, Mixture<D, KC> &m) {
    static_assert(K <= KC, "mixture capacity");
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) s += raw[i * D + k] * raw[i * D + k];
        float inv = s > 0.f ? rsqrtf(s) : 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) m.mu[i * D + k] = s > 0.f ? raw[i * D + k] * inv : (k == 0 ? 1.f : 0.f);
        float kp = fminf(fmaxf(raw[K * D + i], -8.f), 8.f);
        m.kappa[i] = __expf(kp);
        m.lognorm[i] = vmf_lognorm<D>(m.kappa[i]);
    }
    float mx = raw[K * D + K];
#pragma unroll
    for (int i = 1; i < K; ++i) mx = fmaxf(mx, raw[K * D + K + i]);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) { m.lam[i] = __expf(raw[K * D + K + i] - mx); s += m.lam[i]; }
    float inv = 1.f / s;
#pragma unroll
    for (int i = 0; i < K; ++i) m.lam[i] *= inv;
    m.c = 1.f / (1.f + __expf(-raw[K * (D + 2)]));
}

template <int D, int K, int KC>
__device__ __forceinline__ float mixture_pdf(const Mixture<D, KC> &m, const float *nu) {
    float p = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) p += m.lam[i] * __expf(m.lognorm[i] - m.kappa[i] * half_dist2<D>(m.mu + i * D, nu));
    return p;
}

// Best & Fisher (1979) wrapped-Cauchy envelope rejection; the envelope
// parameter rho = (tau - sqrt(2 tau)) / (2 k) is evaluated in a
// cancellation-free form.  Retry j draws from Philox purpose 3 + j (<= 64).
__device__ __forceinline__ float vmf2_angle(float k, uint32_t pid, uint32_t wid, uint32_t step, uint32_t k0,
                                            uint32_t k1) {
    float s = sqrtf(1.f + 4.f * k * k);
    float tau = 1.f + s;
    float rho = 2.f * k * tau / ((s + 1.f) * (tau + sqrtf(2.f * tau)));
    float r = (1.f + rho * rho) / (2.f * rho);
    float f = 0.f, u3 = 0.f;
    for (int j = 0; j < 64; ++j) {
        U4 u = philox(pid, wid, step, P_VMF2 + (uint32_t)j, k0, k1);
        float u1 = u01(u.x), u2 = u01(u.y);
        u3 = u01(u.z);
        float z = cospif(u1);
        f = (1.f + r * z) / (r + z);
        float c = k * (r - f);
        if (c * (2.f - c) - u2 > 0.f) break;
        if (__logf(c / u2) + 1.f - c >= 0.f) break;
    }
    f = fminf(fmaxf(f, -1.f), 1.f);
    float th = acosf(f);
    return u3 < 0.5f ? -th : th;
}

__device__ __forceinline__ void onb3(const float *n, float *b1, float *b2) {
    float sg = n[2] >= 0.f ? 1.f : -1.f;
    float a = -1.f / (sg + n[2]);
    float b = n[0] * n[1] * a;
    b1[0] = 1.f + sg * n[0] * n[0] * a;
    b1[1] = sg * b;
    b1[2] = -sg * n[0];
    b2[0] = b;
    b2[1] = sg + n[1] * n[1] * a;
    b2[2] = -n[1];
}

__device__ __forceinline__ void vmf3_sample(float k, const float *mu, float xi, float xi2, float *nu) {
    float w = 1.f + log1pf(xi * expm1f(-2.f * k)) / k;
    w = fminf(fmaxf(w, -1.f), 1.f);
    float st = sqrtf(fmaxf(0.f, 1.f - w * w));
    float s, c;
    sincospif(2.f * xi2, &s, &c);
    float b1[3], b2[3];
    onb3(mu, b1, b2);
#pragma unroll
    for (int i = 0; i < 3; ++i) nu[i] = w * mu[i] + st * (c * b1[i] + s * b2[i]);
}

// Guided direction (Sec. 4.4 one-sample MIS): with probability c sample the
// mixture (lobe by the lambda-CDF, then a vMF sample), else the uniform
// sphere; the caller reflects below the tangent plane (Sec. 4.3).
// Returns true if the mixture was sampled.
template <int D, int K, int KC>
__device__ __forceinline__ bool sample_direction(const Mixture<D, KC> &m, float c, uint32_t pid, uint32_t wid,
                                                 uint32_t step, uint32_t k0, uint32_t k1, float *nu) {
    U4 u = philox(pid, wid, step, P_MIS, k0, k1);
    if (u01(u.x) < c) {
        // first lobe whose running CDF exceeds u1 (past the end, which
        // rounding allows: the last lobe of nonzero weight)
        float u1 = u01(u.y), cdf = 0.f;
        int lobe = -1;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            cdf += m.lam[i];
            if (u1 < cdf) { lobe = i; break; }
        }
        if (lobe < 0) {
            lobe = K - 1;
            while (lobe > 0 && !(m.lam[lobe] > 0.f)) --lobe;
        }
        const float *mu = m.mu + lobe * D;
        if (D == 2) {
            float th = vmf2_angle(m.kappa[lobe], pid, wid, step, k0, k1);
            float s, cth;
            sincosf(th, &s, &cth);
            nu[0] = mu[0] * cth - mu[1] * s;
            nu[1] = mu[0] * s + mu[1] * cth;
        } else {
            vmf3_sample(m.kappa[lobe], mu, u01(u.z), u01(u.w), nu);
        }
        return true;
    }
    U4 v = philox(pid, wid, step, P_DIR, k0, k1);
    if (D == 2) {
        float s, cth;
        sincospif(2.f * u01(v.x), &s, &cth);
        nu[0] = cth;
        nu[1] = s;
    } else {
        float z = 1.f - 2.f * u01(v.x), s, cth;
        float st = sqrtf(fmaxf(0.f, 1.f - z * z));
        sincospif(2.f * u01(v.y), &s, &cth);
        nu[0] = st * cth;
        nu[1] = st * s;
        nu[2] = z;
    }
    return false;
}

}  // namespace wost

namespace wost {

// ---------------------------------------------------------------------------
// The same direction draw and densities, reading the raw network outputs of
// one walk (FP16, a shared-memory row) lobe by lobe instead of holding the
// whole mixture in registers.  Sampling and density use the same values, so
// the FP16 rounding of the outputs changes the sampler, not its consistency.
// ---------------------------------------------------------------------------
template <int D, int K>
struct RowMixture {
    const __half *y;    // raw outputs (FP16): mu' (K x D), kappa' (K), lambda' (K), c'
    float lam[K];       // normalised mixture weights

    __device__ __forceinline__ float at(int i) const { return __half2float(y[i]); }
    __device__ __forceinline__ void init(const __half *row) {
        y = row;
        float mx = at(K * D + K);
#pragma unroll
        for (int i = 1; i < K; ++i) mx = fmaxf(mx, at(K * D + K + i));
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) { lam[i] = __expf(at(K * D + K + i) - mx); s += lam[i]; }
        float inv = 1.f / s;
#pragma unroll
        for (int i = 0; i < K; ++i) lam[i] *= inv;
    }
    __device__ __forceinline__ float c() const { return 1.f / (1.f + __expf(-at(K * (D + 2)))); }
    __device__ __forceinline__ float kappa(int i) const { return __expf(fminf(fmaxf(at(K * D + i), -8.f), 8.f)); }
    __device__ __forceinline__ void mu(int i, float *m) const {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) { m[k] = at(i * D + k); s += m[k] * m[k]; }
        float inv = s > 0.f ? rsqrtf(s) : 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) m[k] = s > 0.f ? m[k] * inv : (k == 0 ? 1.f : 0.f);
    }
    // density of the mixture at nu (and, if nm != nullptr, plus at nm)
    __device__ __forceinline__ float pdf(const float *nu, const float *nm) const {
        float p = 0.f;
#pragma unroll 1
        for (int i = 0; i < K; ++i) {
            float m[D];
            mu(i, m);
            float k = kappa(i), ln = vmf_lognorm<D>(k);
            float v = __expf(ln - k * half_dist2<D>(m, nu));
            if (nm) v += __expf(ln - k * half_dist2<D>(m, nm));
            p += lam[i] * v;
        }
        return p;
    }
};

template <int D, int K>
__device__ __forceinline__ bool sample_direction_row(const RowMixture<D, K> &m, float c, uint32_t pid, uint32_t wid,
                                                     uint32_t step, uint32_t k0, uint32_t k1, float *nu) {
    U4 u = philox(pid, wid, step, P_MIS, k0, k1);
    if (u01(u.x) < c) {
        // first lobe whose running CDF exceeds u1 (past the end, which
        // rounding allows: the last lobe of nonzero weight)
        float u1 = u01(u.y), cdf = 0.f;
        int lobe = -1;
        for (int i = 0; i < K; ++i) {
            cdf += m.lam[i];
            if (u1 < cdf) { lobe = i; break; }
        }
        if (lobe < 0) {
            lobe = K - 1;
            while (lobe > 0 && !(m.lam[lobe] > 0.f)) --lobe;
        }
        float mu[D];
        m.mu(lobe, mu);
        float k = m.kappa(lobe);
        if (D == 2) {
            float th = vmf2_angle(k, pid, wid, step, k0, k1);
            float s, cth;
            sincosf(th, &s, &cth);
            nu[0] = mu[0] * cth - mu[1] * s;
            nu[1] = mu[0] * s + mu[1] * cth;
        } else {
            vmf3_sample(k, mu, u01(u.z), u01(u.w), nu);
        }
        return true;
    }
    U4 v = philox(pid, wid, step, P_DIR, k0, k1);
    if (D == 2) {
        float s, cth;
        sincospif(2.f * u01(v.x), &s, &cth);
        nu[0] = cth;
        nu[1] = s;
    } else {
        float z = 1.f - 2.f * u01(v.x), s, cth;
        float st = sqrtf(fmaxf(0.f, 1.f - z * z));
        sincospif(2.f * u01(v.y), &s, &cth);
        nu[0] = st * cth;
        nu[1] = st * s;
        nu[2] = z;
    }
    return false;
}

}  // namespace wost

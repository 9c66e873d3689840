// Path contribution f(x) in primary sample space, its log-density
// p = lum(f) + eps, and a hand-written reverse-mode adjoint for grad log p.
//
// The paper samples paths with routines shared by all its methods (Sec. 6,
// "Setup") and differentiates them with Slang's autodiff (Sec. 6); it runs
// MCMC on the full PSS, direct and indirect light together (Sec. 6,
// "Parameter choices").  The sampler here is unidirectional path tracing
// with next-event estimation (one point on one emitting triangle per vertex)
// and balance-heuristic MIS, fixed maximum length L, no Russian roulette.
// PSS layout, d = 2 + 4 (L - 1): x0, x1 = film position (pixel =
// floor(x0 W), floor(x1 H), row 0 at the top); scattering vertex v
// (1 .. L-1) uses base b = 2 + 4 (v - 1): x[b], x[b+1] BSDF sample (first
// coordinate also picks the lobe by rescaling), x[b+2], x[b+3] light sample
// (first coordinate also picks the emitting triangle by rescaling).  f
// carries the pixel importance W H.
//
// The adjoint differentiates the smooth piece containing x: triangle ids,
// lobe choices and visibility are held fixed (what automatic differentiation
// of the sampler gives).  The forward pass records per segment the ray, the
// throughput, the previous BSDF pdf, the hit triangle and the discrete
// choices; the backward pass walks the segments in reverse, recomputes each
// vertex from its ray and triangle (no traversal), and applies the
// vector-Jacobian products of each step.
#pragma once
#include "dr_trace.cuh"

namespace dr {

// ---------------------------------------------------------------- records
struct MatP {
  int type;
  bool cond;  // a conductor; constant false in code built without conductor support
  float3 albedo, emit;  // conductor: albedo = eta; k at rec[9..11]
  const float* rec;
  float rough, ior, f0;
  bool emissive;
};

// COND = false: the caller's scene has no conductor, and the conductor
// branches are compiled out of the kernel.
template <bool COND = true>
DR_D MatP load_mat(const float* __restrict__ mats, int id) {
  const float* m = mats + kMatFloats * id;
  MatP r;
  r.type = (int)__ldg(m + 0);
  r.cond = COND && r.type == kConductor;
  r.albedo = f3(__ldg(m + 1), __ldg(m + 2), __ldg(m + 3));
  r.rough = __ldg(m + 4);
  r.ior = __ldg(m + 5);
  r.emit = f3(__ldg(m + 6), __ldg(m + 7), __ldg(m + 8));
  r.f0 = __ldg(m + 9);
  r.rec = m;
  r.emissive = r.emit.x > 0.f || r.emit.y > 0.f || r.emit.z > 0.f;
  return r;
}

struct Surf {
  float3 v0, N, ng, au, av;
  float area, sel;
  int mat;
  bool has_n;
};

DR_D Surf load_surf(const DevScene& S, int tri) {
  const float4 a = __ldg(S.surf + kSurfF4 * tri + 0);
  const float4 b = __ldg(S.surf + kSurfF4 * tri + 1);
  const float4 c = __ldg(S.surf + kSurfF4 * tri + 2);
  const float4 d = __ldg(S.surf + kSurfF4 * tri + 3);
  const float4 e = __ldg(S.surf + kSurfF4 * tri + 4);
  Surf s;
  s.v0 = xyz(a);
  s.mat = __float_as_int(a.w);
  s.N = xyz(b);
  s.area = b.w;
  s.ng = xyz(c);
  s.au = xyz(d);
  s.sel = d.w;
  s.av = xyz(e);
  s.has_n = S.nrm != nullptr && (__float_as_int(c.w) & 1);
  return s;
}

DR_D void load_vnormals(const DevScene& S, int tri, float3& n0, float3& n1, float3& n2) {
  const float* p = S.nrm + 9 * tri;
  n0 = f3(__ldg(p + 0), __ldg(p + 1), __ldg(p + 2));
  n1 = f3(__ldg(p + 3), __ldg(p + 4), __ldg(p + 5));
  n2 = f3(__ldg(p + 6), __ldg(p + 7), __ldg(p + 8));
}

// Asks for the triangle's vertex normals (36 B) to be brought into L1, so
// that the load in shading_normal, issued behind the branches that need the
// material, finds them there.  Holds no registers.
DR_D void prefetch_vnormals(const DevScene& S, int tri, const Surf& sf) {
  if (!sf.has_n) return;
  const float* p = S.nrm + 9 * tri;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p + 8));
}

// Interpolated, normalised shading normal at P (un-flipped) and its raw sum.
DR_D float3 shading_normal(const DevScene& S, int tri, const Surf& sf, float3 P, float3* raw_out) {
  if (!sf.has_n) {
    *raw_out = sf.ng;
    return sf.ng;
  }
  float3 n0, n1, n2;
  load_vnormals(S, tri, n0, n1, n2);
  const float3 q = P - sf.v0;
  const float bu = dot(q, sf.au), bv = dot(q, sf.av);
  const float3 raw = n0 * (1.0f - bu - bv) + n1 * bu + n2 * bv;
  *raw_out = raw;
  return normalize(raw);
}

DR_D float3 shading_normal_bwd(const DevScene& S, int tri, const Surf& sf, float3 raw, float3 nsn, float3 gnsn) {
  if (!sf.has_n) return f3(0.f, 0.f, 0.f);
  float3 n0, n1, n2;
  load_vnormals(S, tri, n0, n1, n2);
  const float3 graw = normalize_bwd(raw, nsn, gnsn);
  const float gbu = dot(graw, n1 - n0), gbv = dot(graw, n2 - n0);
  return sf.au * gbu + sf.av * gbv;
}

// ---------------------------------------------------------------- basis
// Orthonormal basis around unit n (Duff et al. 2017, branchless form).
DR_D void onb(float3 n, float3& t, float3& b) {
  const float s = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (s + n.z);
  const float c = n.x * n.y * a;
  t = f3(1.0f + s * n.x * n.x * a, s * c, -s * n.x);
  b = f3(c, s + n.y * n.y * a, -n.y);
}

DR_D float3 onb_bwd(float3 n, float3 gt, float3 gb) {
  const float s = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (s + n.z);
  const float gc = gt.y * s + gb.x;
  const float ga = gt.x * s * n.x * n.x + gb.y * n.y * n.y + gc * n.x * n.y;
  float3 g;
  g.x = gt.x * 2.0f * s * n.x * a - gt.z * s + gc * n.y * a;
  g.y = gb.y * 2.0f * n.y * a - gb.z + gc * n.x * a;
  g.z = ga * a * a;
  return g;
}

// ---------------------------------------------------------------- BSDFs
// GGX (Trowbridge-Reitz) D, Smith height-correlated G2.  The glossy BSDF is
// a GGX coat (Schlick F) over a Lambertian base, sampled by picking the
// specular lobe with probability 1/2 (D cos(theta_h) half-vector sampling)
// or the cosine-weighted diffuse lobe; its pdf is the two-lobe mixture.  The
// rough conductor (pbrt's conductor, Sec. 6 "Test scenes") is the specular
// lobe alone with the Fresnel reflectance of a complex index per channel,
// always sampled by half-vectors.
struct GlossyFwd {
  float co, ci, hl, nh, oh, ih, k, D, lo, li, ro, ri, G, pdf, sp;
  float3 h, hv;
};

DR_D float spec_prob(const MatP& m) { return m.cond ? 1.0f : kGlossySpecProb; }
DR_D float spec_prob_inv(const MatP& m) { return m.cond ? 1.0f : 1.0f / kGlossySpecProb; }

DR_D GlossyFwd glossy_fwd(const MatP& m, float3 n, float3 wo, float3 wi) {
  GlossyFwd g;
  const float a2 = m.rough * m.rough;
  g.sp = spec_prob(m);
  g.co = dot(n, wo);
  g.ci = dot(n, wi);
  g.hv = wo + wi;
  g.hl = sqrtf(dot(g.hv, g.hv));
  g.h = g.hv * (1.0f / g.hl);
  g.nh = dot(n, g.h);
  g.oh = dot(wo, g.h);
  g.ih = dot(wi, g.h);
  g.k = g.nh * g.nh * (a2 - 1.0f) + 1.0f;
  g.D = a2 / (kPi * g.k * g.k);
  g.ro = sqrtf(1.0f + a2 * (1.0f - g.co * g.co) / (g.co * g.co));
  g.ri = sqrtf(1.0f + a2 * (1.0f - g.ci * g.ci) / (g.ci * g.ci));
  g.lo = 0.5f * (g.ro - 1.0f);
  g.li = 0.5f * (g.ri - 1.0f);
  g.G = 1.0f / (1.0f + g.lo + g.li);
  g.pdf = g.sp * g.D * g.nh / (4.0f * fabsf(g.oh)) + (1.0f - g.sp) * g.ci * kInvPi;
  return g;
}

// Fresnel reflectance of unpolarised light from vacuum onto an interface of
// complex index eta + i k, written in real variables: with
// A = |(eta + i k)^2 - sin^2| and a = sqrt((A + Re) / 2),
// R_s = (A + c^2 - 2ac) / (A + c^2 + 2ac) and
// R_p = R_s (c^2 A + s^4 - 2ac s^2) / (c^2 A + s^4 + 2ac s^2); R = (R_s + R_p) / 2.
// Also returns dR/dc (forward-mode, for the adjoint).
DR_D float fresnel_conductor(float c, float eta, float k, float* dFdc) {
  const float c2 = c * c, s2 = 1.0f - c2, ds2 = -2.0f * c;
  const float t0 = eta * eta - k * k - s2, dt0 = -ds2;
  const float A = sqrtf(t0 * t0 + 4.0f * eta * eta * k * k), dA = t0 * dt0 / A;
  const float a = sqrtf(fmaxf(0.5f * (A + t0), 0.0f));
  const float da = a > 0.0f ? (dA + dt0) / (4.0f * a) : 0.0f;
  const float t1 = A + c2, dt1 = dA + 2.0f * c;
  const float t2 = 2.0f * a * c, dt2 = 2.0f * (da * c + a);
  const float q1 = 1.0f / (t1 + t2);
  const float Rs = (t1 - t2) * q1;
  const float dRs = 2.0f * (t2 * dt1 - t1 * dt2) * q1 * q1;
  const float t3 = c2 * A + s2 * s2, dt3 = 2.0f * c * A + c2 * dA + 2.0f * s2 * ds2;
  const float t4 = t2 * s2, dt4 = dt2 * s2 + t2 * ds2;
  const float q2 = 1.0f / (t3 + t4);
  const float Q = (t3 - t4) * q2;
  const float dQ = 2.0f * (t4 * dt3 - t3 * dt4) * q2 * q2;
  *dFdc = 0.5f * (dRs * (1.0f + Q) + Rs * dQ);
  return 0.5f * Rs * (1.0f + Q);
}

// Per-channel Fresnel of the specular lobe at cos = ih.
DR_D float3 lobe_fresnel(const MatP& m, float ih) {
  if (m.cond) {
    // k is read here rather than with the record: it is live only here
    float d;
    return f3(fresnel_conductor(ih, m.albedo.x, __ldg(m.rec + 9), &d),
              fresnel_conductor(ih, m.albedo.y, __ldg(m.rec + 10), &d),
              fresnel_conductor(ih, m.albedo.z, __ldg(m.rec + 11), &d));
  }
  const float om = 1.0f - ih, om2 = om * om;
  const float F = m.f0 + (1.0f - m.f0) * (om2 * om2 * om);
  return f3(F, F, F);
}

// sum_c g_c F_c and sum_c g_c dF_c/d(ih) for the adjoint, one channel at a
// time (few live registers).
DR_D void lobe_fresnel_dots(const MatP& m, float ih, float3 g, float* gF, float* gdF) {
  if (m.cond) {
    float d0, d1, d2;
    const float F0 = fresnel_conductor(ih, m.albedo.x, __ldg(m.rec + 9), &d0);
    float sF = g.x * F0, sd = g.x * d0;
    const float F1 = fresnel_conductor(ih, m.albedo.y, __ldg(m.rec + 10), &d1);
    sF += g.y * F1;
    sd += g.y * d1;
    const float F2 = fresnel_conductor(ih, m.albedo.z, __ldg(m.rec + 11), &d2);
    *gF = sF + g.z * F2;
    *gdF = sd + g.z * d2;
    return;
  }
  const float om = 1.0f - ih, om2 = om * om;
  const float F = m.f0 + (1.0f - m.f0) * (om2 * om2 * om);
  const float gs = g.x + g.y + g.z;
  *gF = gs * F;
  *gdF = gs * (-5.0f * (1.0f - m.f0) * om2 * om2);
}

// BSDF value (RGB) and sampling pdf (solid angle) of an opaque material.
DR_D float3 bsdf_eval(const MatP& m, float3 n, float3 wo, float3 wi, float* pdf) {
  if (m.type == kGlossy || m.cond) {
    const GlossyFwd g = glossy_fwd(m, n, wo, wi);
    *pdf = g.pdf;
    const float DG = g.D * g.G, den = 4.0f * g.co * g.ci;
    if (m.cond) return lobe_fresnel(m, g.ih) * (DG / den);
    const float spec = DG * lobe_fresnel(m, g.ih).x / den;
    const float kd = (1.0f - m.f0) * kInvPi;
    return m.albedo * kd + f3(spec, spec, spec);
  }
  *pdf = dot(n, wi) * kInvPi;
  return m.albedo * kInvPi;
}

// Backward of bsdf_eval: given d(fs) (RGB) and d(pdf), accumulates into
// d(n), d(wo), d(wi).
DR_D void bsdf_eval_bwd(const MatP& m, float3 n, float3 wo, float3 wi, float3 gfs, float gpdf, float3& gn,
                        float3& gwo, float3& gwi) {
  if (m.type != kGlossy && !m.cond) {
    gn += wi * (gpdf * kInvPi);
    gwi += n * (gpdf * kInvPi);
    return;
  }
  const GlossyFwd g = glossy_fwd(m, n, wo, wi);
  float gFsum, gdF;  // sum_c gfs_c F_c, sum_c gfs_c dF_c / d(ih)
  lobe_fresnel_dots(m, g.ih, gfs, &gFsum, &gdF);
  const float a2 = m.rough * m.rough;
  const float den = 4.0f * g.co * g.ci;
  const float aoh = fabsf(g.oh);
  const float gspec = gFsum * (g.D * g.G / den);  // sum_c gfs_c spec_c
  const float gD = gFsum * g.G / den + gpdf * g.sp * g.nh / (4.0f * aoh);
  const float gG = gFsum * g.D / den;
  // Lambda'(c) = -a2 / (2 r c^3), dG/dLambda = -G^2
  const float dlo = -a2 / (2.0f * g.ro * g.co * g.co * g.co);
  const float dli = -a2 / (2.0f * g.ri * g.ci * g.ci * g.ci);
  const float gco = -gspec / g.co - gG * g.G * g.G * dlo;
  const float gci = -gspec / g.ci - gG * g.G * g.G * dli + gpdf * (1.0f - g.sp) * kInvPi;
  const float dD = g.D * (-4.0f * g.nh * (a2 - 1.0f) / g.k);
  const float gnh = gD * dD + gpdf * g.sp * g.D / (4.0f * aoh);
  const float goh = -gpdf * g.sp * g.D * g.nh * (g.oh >= 0.0f ? 1.0f : -1.0f) / (4.0f * g.oh * g.oh);
  const float gih = gdF * (g.D * g.G / den);
  const float3 gh = n * gnh + wo * goh + wi * gih;
  gn += g.h * gnh;
  gwo += g.h * goh;
  gwi += g.h * gih;
  const float3 ghv = (gh - g.h * dot(g.h, gh)) * (1.0f / g.hl);
  gwo += ghv;
  gwi += ghv;
  gn += wo * gco + wi * gci;
  gwo += n * gco;
  gwi += n * gci;
}

// Cosine-weighted direction (local frame) and its backward.
DR_D float3 cosine_local(float u, float u2, float* r, float* cph, float* sph) {
  *r = sqrtf(u);
  sincospif(2.0f * u2, sph, cph);
  return f3(*r * *cph, *r * *sph, sqrtf(1.0f - u));
}

struct SampleRec {
  float3 wi;
  float3 w;
  float pdf;
  int lobe;
};

// BSDF sampling of an opaque material at a vertex with shading normal n,
// geometric normal ngf (same side as wo).  Returns false if wi is not above
// both normals.
DR_D bool opaque_sample(const MatP& m, float3 n, float3 ngf, float3 wo, float u1, float u2, SampleRec& s) {
  float3 t, b;
  onb(n, t, b);
  if ((m.type == kGlossy && u1 < kGlossySpecProb) || m.cond) {
    s.lobe = 1;
    const float v = u1 * spec_prob_inv(m);
    const float a2 = m.rough * m.rough;
    const float den = 1.0f + (a2 - 1.0f) * v;
    const float ch = sqrtf((1.0f - v) / den);
    const float sh = m.rough * sqrtf(v / den);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float3 h = t * (sh * cp) + b * (sh * sp) + n * ch;
    s.wi = h * (2.0f * dot(wo, h)) - wo;
  } else {
    s.lobe = 0;
    const float v = m.type == kGlossy ? (u1 - kGlossySpecProb) * (1.0f / (1.0f - kGlossySpecProb)) : u1;
    float r, cp, sp;
    const float3 l = cosine_local(v, u2, &r, &cp, &sp);
    s.wi = t * l.x + b * l.y + n * l.z;
  }
  const float ci = dot(n, s.wi);
  if (!(ci > 0.0f) || !(dot(ngf, s.wi) > 0.0f)) return false;
  const float3 fs = bsdf_eval(m, n, wo, s.wi, &s.pdf);
  s.w = fs * (ci / s.pdf);
  return true;
}

// Backward of the sampled direction wi(n, wo, u1, u2) for the recorded lobe.
DR_D void opaque_sample_dir_bwd(const MatP& m, int lobe, float3 n, float3 wo, float u1, float u2, float3 gwi,
                                float3& gn, float3& gwo, float& gu1, float& gu2) {
  float3 t, b;
  onb(n, t, b);
  float3 gt, gb;
  if (lobe == 1) {
    const float pinv = spec_prob_inv(m);
    const float v = u1 * pinv;
    const float a2 = m.rough * m.rough;
    const float den = 1.0f + (a2 - 1.0f) * v;
    const float ch = sqrtf((1.0f - v) / den);
    const float sh = m.rough * sqrtf(v / den);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float3 h = t * (sh * cp) + b * (sh * sp) + n * ch;
    const float oh = dot(wo, h);
    const float wh = dot(gwi, h);
    const float3 gh = gwi * (2.0f * oh) + wo * (2.0f * wh);
    gwo += h * (2.0f * wh) - gwi;
    gt = gh * (sh * cp);
    gb = gh * (sh * sp);
    gn += gh * ch;
    const float ght = dot(gh, t), ghb = dot(gh, b);
    const float gsh = ght * cp + ghb * sp;
    const float gch = dot(gh, n);
    const float gph = sh * (-sp * ght + cp * ghb);
    const float den2 = den * den;
    float gv = 0.0f;
    if (sh > 0.0f) gv += gsh * a2 / (2.0f * sh * den2);
    if (ch > 0.0f) gv -= gch * a2 / (2.0f * ch * den2);
    gu1 = gv * pinv;
    gu2 = gph * 2.0f * kPi;
  } else {
    const float dvdu = m.type == kGlossy ? 1.0f / (1.0f - kGlossySpecProb) : 1.0f;
    const float v = m.type == kGlossy ? (u1 - kGlossySpecProb) * dvdu : u1;
    float r, cp, sp;
    const float3 l = cosine_local(v, u2, &r, &cp, &sp);
    const float glx = dot(gwi, t), gly = dot(gwi, b), glz = dot(gwi, n);
    gt = gwi * l.x;
    gb = gwi * l.y;
    gn += gwi * l.z;
    float gv = 0.0f;
    if (r > 0.0f) gv += (glx * cp + gly * sp) / (2.0f * r);
    if (l.z > 0.0f) gv -= glz / (2.0f * l.z);
    gu1 = gv * dvdu;
    gu2 = r * (-glx * sp + gly * cp) * 2.0f * kPi;
  }
  gn += onb_bwd(n, gt, gb);
}

// Exact dielectric Fresnel reflectance, eta = n_t / n_i.
DR_D float fresnel_dielectric(float ci, float ct, float eta) {
  const float rs = (ci - eta * ct) / (ci + eta * ct);
  const float rp = (eta * ci - ct) / (eta * ci + ct);
  return 0.5f * (rs * rs + rp * rp);
}

// ---------------------------------------------------------------- tape
enum : int {
  kFPrevDelta = 1 << 0,
  kFNeeVis = 1 << 1,
  kFScatter = 1 << 2,   // BSDF sample succeeded (next segment traced)
  kFLobeShift = 3,      // 2 bits: 0 diffuse, 1 glossy spec, 2 reflect, 3 refract
  kFLightShift = 8,
};

template <int LMAX>
struct Tape {
  float4 a[LMAX];  // (o, prev pdf)
  float4 b[LMAX];  // (d, tri bits)
  float4 c[LMAX];  // (beta, flags bits)
};

struct PathResult {
  float3 f;
  int pix;
  int nseg;
  uint32_t rays;
};

DR_D int pixel_of(float x0, float x1, int W, int H) {
  int col = (int)floorf(x0 * (float)W), row = (int)floorf(x1 * (float)H);
  col = min(max(col, 0), W - 1);
  row = min(max(row, 0), H - 1);
  return row * W + col;
}

// A hit is kept when the unit ray direction is not within 1e-6 (cosine) of
// the triangle's plane.
DR_D bool grazing_ok(float3 d, float3 ng) { return fabsf(dot(d, ng)) >= 1e-6f; }

DR_D float3 camera_dir(const Camera& C, float x0, float x1, float3* raw) {
  const float sx = (2.0f * x0 - 1.0f) * C.tx, sy = (1.0f - 2.0f * x1) * C.ty;
  *raw = C.fwd + C.right * sx + C.up * sy;
  return normalize(*raw);
}

// Light pick by the first light coordinate (CDF over emitting triangles,
// prefix of area * lum(emission)), rescaled to [0, 1).
DR_D int pick_light(const DevScene& S, float ul, float* lo, float* pk) {
  int a = 0, b = S.n_lights - 1;
  while (a < b) {  // first k with ul < cdf[k]
    const int mid = (a + b) >> 1;
    if (ul < __ldg(&S.lights[kLightF4 * mid + 3].x)) b = mid; else a = mid + 1;
  }
  *lo = a == 0 ? 0.0f : __ldg(&S.lights[kLightF4 * (a - 1) + 3].x);
  *pk = __ldg(&S.lights[kLightF4 * a + 3].x) - *lo;
  return a;
}

struct LightSample {
  float3 V0, V1, V2, nl, y, Le;
  float v1, v2, su, sel, area, pk;
  int tri;
  bool clamped;
};

DR_D LightSample light_sample(const DevScene& S, int k, float ul, float ul2, float lo, float pk) {
  LightSample ls;
  const float4 l0 = __ldg(S.lights + kLightF4 * k + 0);
  const float4 l1 = __ldg(S.lights + kLightF4 * k + 1);
  const float4 l2 = __ldg(S.lights + kLightF4 * k + 2);
  ls.V0 = xyz(l0);
  ls.V1 = xyz(l1);
  ls.V2 = xyz(l2);
  ls.tri = __float_as_int(l0.w);
  ls.sel = l1.w;
  ls.area = l2.w;
  ls.pk = pk;
  float v1 = (ul - lo) / pk;
  ls.clamped = false;
  if (v1 >= 1.0f) { v1 = 0.99999994f; ls.clamped = true; }
  if (v1 < 0.0f) { v1 = 0.0f; ls.clamped = true; }
  ls.v1 = v1;
  ls.v2 = ul2;
  ls.su = sqrtf(v1);
  ls.y = ls.V0 * (1.0f - ls.su) + ls.V1 * (ls.su * (1.0f - ul2)) + ls.V2 * (ls.su * ul2);
  ls.nl = normalize(cross(ls.V1 - ls.V0, ls.V2 - ls.V0));
  const float4 l3 = __ldg(S.lights + kLightF4 * k + 3);  // the emission rides in the light record
  ls.Le = f3(l3.y, l3.z, l3.w);
  return ls;
}

// Tape accessors: a per-thread array, or a [segment][3][N] float4 array in
// global memory (wavefront execution), or nothing.
template <int LMAX>
struct LocalTape {
  Tape<LMAX>* t;
  DR_D void put(int s, float4 a, float4 b, float4 c) const { t->a[s] = a; t->b[s] = b; t->c[s] = c; }
  DR_D void set_flags(int s, int f) const { t->c[s].w = __int_as_float(f); }
  DR_D void or_flags(int s, int f) const { t->c[s].w = __int_as_float(__float_as_int(t->c[s].w) | f); }
  DR_D void get(int s, float4& a, float4& b, float4& c) const { a = t->a[s]; b = t->b[s]; c = t->c[s]; }
};

struct GlobalTape {
  float4* base;
  unsigned long long N, j;
  DR_D float4* at(int s, int k) const { return base + ((size_t)s * 3 + k) * N + j; }
  DR_D void put(int s, float4 a, float4 b, float4 c) const { *at(s, 0) = a; *at(s, 1) = b; *at(s, 2) = c; }
  DR_D void set_flags(int s, int f) const { at(s, 2)->w = __int_as_float(f); }
  DR_D void or_flags(int s, int f) const { at(s, 2)->w = __int_as_float(__float_as_int(at(s, 2)->w) | f); }
  DR_D void get(int s, float4& a, float4& b, float4& c) const { a = *at(s, 0); b = *at(s, 1); c = *at(s, 2); }
};

struct NoTape {
  DR_D void put(int, float4, float4, float4) const {}
  DR_D void set_flags(int, int) const {}
  DR_D void or_flags(int, int) const {}
};

// State of one path between segments.
struct PathState {
  float3 o, d, beta, f;
  float ppdf;
  int prev_tri, prev_delta, nseg;
};

// Next-event estimation request of one vertex: the shadow ray and the
// contribution that is added to f if the ray is unoccluded.
struct NeeReq {
  float3 o, wi, contrib;
  float tmax;
  int ex0, ex1, seg;
  bool valid;
};

// Camera ray from the film pair; returns the pixel.
template <class XA>
DR_D int path_begin(const DevScene& S, const XA& xa, PathState& ps) {
  const float WH = (float)S.W * (float)S.H;
  ps.beta = f3(WH, WH, WH);
  ps.f = f3(0.f, 0.f, 0.f);
  const float x0 = xa(0), x1 = xa(1);
  float3 raw;
  ps.d = camera_dir(S.cam, x0, x1, &raw);
  ps.o = S.cam.eye;
  ps.prev_tri = -1;
  ps.prev_delta = 1;
  ps.ppdf = 0.0f;
  ps.nseg = 0;
  return pixel_of(x0, x1, S.W, S.H);
}

// Processes the closest hit `tri` of segment `seg` (1-based): records the
// tape entry, adds the hit's emission (MIS-weighted after a non-delta
// vertex), prepares the NEE request of the vertex and samples the next
// direction.  Returns whether the path continues (ps then holds the next
// ray).  The NEE contribution is added by the caller once the shadow ray
// is found unoccluded, before the next vertex.
template <bool COND = true, class XA, class TP>
DR_D bool path_vertex(const DevScene& S, const XA& xa, int L, int seg, int tri, PathState& ps, const TP& tape,
                      NeeReq& nee) {
  nee.valid = false;
  // The vertex's coordinates are loaded with the surface record, and the
  // vertex normals are asked for as soon as that record is in, ahead of the
  // branches that use them: fewer rounds of memory latency per vertex.
  const Surf sf = load_surf(S, tri);
  const int b = 2 + 4 * (seg - 1);
  float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f, u3 = 0.0f;  // x_b .. x_{b+3}; a vertex at seg == L has none
  if (seg < L) {
    u0 = xa(b);
    u1 = xa(b + 1);
    u2 = xa(b + 2);
    u3 = xa(b + 3);
  }
  prefetch_vnormals(S, tri, sf);
  // grazing hits (|cos| < 1e-6) end the path: the differentiable hit
  // distance (v0 - o).N / d.N is ill-conditioned there
  if (!grazing_ok(ps.d, sf.ng)) return false;
  ps.nseg = seg;
  int flags = ps.prev_delta ? kFPrevDelta : 0;
  tape.put(seg - 1, make_float4(ps.o.x, ps.o.y, ps.o.z, ps.ppdf), make_float4(ps.d.x, ps.d.y, ps.d.z, __int_as_float(tri)),
           make_float4(ps.beta.x, ps.beta.y, ps.beta.z, __int_as_float(flags)));
  const MatP m = load_mat<COND>(S.mats, sf.mat);
  const float t = dot(sf.v0 - ps.o, sf.N) / dot(ps.d, sf.N);
  const float3 P = ps.o + ps.d * t;
  if (m.emissive) {
    const float cl = -dot(sf.ng, ps.d);
    if (cl > 0.0f) {
      float w = 1.0f;
      if (!ps.prev_delta) {
        const float pl = sf.sel / sf.area * t * t / cl;
        w = ps.ppdf / (ps.ppdf + pl);
      }
      ps.f += ps.beta * m.emit * w;
    }
  }
  if (m.type == kEmitter || seg == L) return false;
  const float3 wo = -ps.d;
  float3 nraw;
  float3 ns = shading_normal(S, tri, sf, P, &nraw);
  if (m.type == kDielectric) {
    const bool entering = dot(sf.ng, wo) > 0.0f;
    const float3 nn = entering ? ns : -ns;
    const float c = dot(nn, wo);
    if (!(c > 0.0f)) return false;
    const float eta = entering ? m.ior : 1.0f / m.ior;
    const float s2 = (1.0f - c * c) / (eta * eta);
    float F = 1.0f, ct = 0.0f;
    if (s2 < 1.0f) {
      ct = sqrtf(1.0f - s2);
      F = fresnel_dielectric(c, ct, eta);
    }
    float3 wi;
    float wgt;
    int lobe;
    if (u0 < F) {
      wi = nn * (2.0f * c) - wo;
      wgt = 1.0f;
      lobe = 2;
    } else {
      wi = wo * (-1.0f / eta) + nn * (c / eta - ct);
      wgt = 1.0f / (eta * eta);
      lobe = 3;
    }
    ps.beta = ps.beta * wgt;
    flags |= kFScatter | (lobe << kFLobeShift);
    tape.set_flags(seg - 1, flags);
    ps.prev_delta = 1;
    ps.ppdf = 0.0f;
    ps.o = P;
    ps.d = wi;
    ps.prev_tri = tri;
    return true;
  }
  float3 ngf = sf.ng;
  if (dot(ngf, wo) < 0.0f) {
    ngf = -ngf;
    ns = -ns;
  }
  if (!(dot(ns, wo) > 0.0f)) return false;
  if (S.n_lights > 0) {
    float lo, pk;
    const int k = pick_light(S, u2, &lo, &pk);
    flags |= k << kFLightShift;
    const LightSample ls = light_sample(S, k, u2, u3, lo, pk);
    const float3 wv = ls.y - P;
    const float dist2 = dot(wv, wv);
    const float dist = sqrtf(dist2);
    const float3 wi = wv * (1.0f / dist);
    const float ci = dot(ns, wi);
    const float cl = -dot(ls.nl, wi);
    if (ci > 0.0f && cl > 0.0f && dot(ngf, wi) > 0.0f) {
      float pb;
      const float3 fs = bsdf_eval(m, ns, wo, wi, &pb);
      const float pl = ls.sel / ls.area * dist2 / cl;
      const float g = ci / (pl + pb);
      nee.valid = true;
      nee.o = P;
      nee.wi = wi;
      nee.tmax = dist - S.tmin;
      nee.ex0 = tri;
      nee.ex1 = ls.tri;
      nee.seg = seg;
      nee.contrib = ps.beta * fs * ls.Le * g;
    }
  }
  SampleRec s;
  const bool ok = opaque_sample(m, ns, ngf, wo, u0, u1, s);
  if (ok) flags |= kFScatter | (s.lobe << kFLobeShift);
  tape.set_flags(seg - 1, flags);
  if (!ok) return false;
  ps.beta = ps.beta * s.w;
  ps.prev_delta = 0;
  ps.ppdf = s.pdf;
  ps.o = P;
  ps.d = s.wi;
  ps.prev_tri = tri;
  return true;
}

// Forward path evaluation in one thread (traversal inline).  XA: functor
// x(i) -> float.  With TAPE the per-segment record for the adjoint is
// written to *tape.
template <int STACK, bool STATS, bool TAPE, bool COND = true, int LMAX, class XA>
DR_D PathResult path_forward(const DevScene& S, const XA& xa, int L, Tape<LMAX>* tape, TraceStack<STACK> st,
                             uint32_t* err, TraceStats* stats) {
  PathResult res;
  res.rays = 0;
  PathState ps;
  res.pix = path_begin(S, xa, ps);
  for (int seg = 1; seg <= L; ++seg) {
    ++res.rays;
    float th;
    const int tri = trace_closest<STACK, STATS>(S, make_ray(ps.o, ps.d), ps.prev_tri, &th, st, err, stats);
    if (tri < 0) break;
    NeeReq nee;
    bool cont;
    if (TAPE) cont = path_vertex<COND>(S, xa, L, seg, tri, ps, LocalTape<LMAX>{tape}, nee);
    else cont = path_vertex<COND>(S, xa, L, seg, tri, ps, NoTape{}, nee);
    if (nee.valid) {
      ++res.rays;
      if (!trace_any<STACK, STATS>(S, make_ray(nee.o, nee.wi), nee.tmax, nee.ex0, nee.ex1, st, err, stats)) {
        ps.f += nee.contrib;
        if (TAPE) LocalTape<LMAX>{tape}.or_flags(seg - 1, kFNeeVis);
      }
    }
    if (!cont) break;
  }
  res.f = ps.f;
  res.nseg = ps.nseg;
  return res;
}

// Reverse-mode adjoint of p = lum(f) + eps with respect to x, using the tape
// of a forward pass with the same x.  GW: functor gw(i, value) receiving
// d log p / d x_i = (d p / d x_i) / p; every i < d is written exactly once.
template <bool COND = true, class TP, class XA, class GW>
DR_D void path_adjoint(const DevScene& S, const XA& xa, int L, float p, const TP& tape, int nseg, const GW& gw) {
  const float inv_p = 1.0f / p;
  const float3 lw = lum_weights();
  float3 go = f3(0.f, 0.f, 0.f), gd = f3(0.f, 0.f, 0.f), gbeta = f3(0.f, 0.f, 0.f);
  float gpp = 0.0f;
  // vertices that were never reached have zero gradient
  for (int v = L - 1; v > nseg; --v) {
    const int b = 2 + 4 * (v - 1);
    gw(b, 0.f); gw(b + 1, 0.f); gw(b + 2, 0.f); gw(b + 3, 0.f);
  }
  for (int seg = nseg; seg >= 1; --seg) {
    float4 ta, tb, tc;
    tape.get(seg - 1, ta, tb, tc);
    const float3 o = xyz(ta), d = xyz(tb), beta = xyz(tc);
    const float ppdf = ta.w;
    const int tri = __float_as_int(tb.w);
    const int flags = __float_as_int(tc.w);
    const bool prev_delta = flags & kFPrevDelta;
    const Surf sf = load_surf(S, tri);
    const MatP m = load_mat<COND>(S.mats, sf.mat);
    const float dn = dot(d, sf.N);
    const float t = dot(sf.v0 - o, sf.N) / dn;
    const float3 P = o + d * t;
    float3 gP = f3(0.f, 0.f, 0.f), gdd = f3(0.f, 0.f, 0.f), gbb = f3(0.f, 0.f, 0.f);
    float gt = 0.0f, gppd = 0.0f;
    // emission at this hit
    if (m.emissive) {
      const float cl = -dot(sf.ng, d);
      if (cl > 0.0f) {
        float w = 1.0f;
        if (!prev_delta) {
          const float pl = sf.sel / sf.area * t * t / cl;
          const float den = ppdf + pl;
          w = ppdf / den;
          const float gw_ = dot(lw * beta, m.emit);
          gppd += gw_ * pl / (den * den);
          const float gpl = -gw_ * ppdf / (den * den);
          gt += gpl * 2.0f * pl / t;
          const float gcl = -gpl * pl / cl;
          gdd += sf.ng * (-gcl);
        }
        gbb += lw * m.emit * w;
      }
    }
    const int b = 2 + 4 * (seg - 1);
    const bool vertex = !(m.type == kEmitter || seg == L);
    if (vertex) {
      const float3 wo = -d;
      float3 gwo = f3(0.f, 0.f, 0.f), gns = f3(0.f, 0.f, 0.f);
      float3 nraw;
      const float3 nsn = shading_normal(S, tri, sf, P, &nraw);
      float sgn = 1.0f;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
      const int lobe = (flags >> kFLobeShift) & 3;
      if (m.type == kDielectric) {
        const bool entering = dot(sf.ng, wo) > 0.0f;
        sgn = entering ? 1.0f : -1.0f;
        const float3 nn = nsn * sgn;
        if (flags & kFScatter) {
          const float c = dot(nn, wo);
          const float eta = entering ? m.ior : 1.0f / m.ior;
          const float wgt = lobe == 2 ? 1.0f : 1.0f / (eta * eta);
          gbb += gbeta * wgt;
          gP += go;
          float3 gnn = f3(0.f, 0.f, 0.f);
          float gc;
          if (lobe == 2) {
            gc = 2.0f * dot(gd, nn);
            gnn += gd * (2.0f * c);
            gwo -= gd;
          } else {
            const float ct = sqrtf(fmaxf(0.0f, 1.0f - (1.0f - c * c) / (eta * eta)));
            const float k = c / eta - ct;
            const float gk = dot(gd, nn);
            gnn += gd * k;
            gwo += gd * (-1.0f / eta);
            gc = gk * (1.0f / eta - (ct > 0.0f ? c / (eta * eta * ct) : 0.0f));
          }
          gnn += wo * gc;
          gwo += nn * gc;
          gns += gnn;  // in the frame of nn; mapped to nsn below via sgn
        }
      } else {
        float3 ngf = sf.ng;
        if (dot(ngf, wo) < 0.0f) {
          ngf = -ngf;
          sgn = -1.0f;
        }
        const float3 ns = nsn * sgn;
        if (flags & kFNeeVis) {
          const int k = flags >> kFLightShift;
          float lo = k == 0 ? 0.0f : __ldg(&S.lights[kLightF4 * (k - 1) + 3].x);
          const float pk = __ldg(&S.lights[kLightF4 * k + 3].x) - lo;
          const LightSample ls = light_sample(S, k, xa(b + 2), xa(b + 3), lo, pk);
          const float3 wv = ls.y - P;
          const float dist2 = dot(wv, wv);
          const float dist = sqrtf(dist2);
          const float3 wi = wv * (1.0f / dist);
          const float ci = dot(ns, wi);
          const float cl = -dot(ls.nl, wi);
          float pb;
          const float3 fs = bsdf_eval(m, ns, wo, wi, &pb);
          const float pl = ls.sel / ls.area * dist2 / cl;
          const float den = pl + pb;
          const float g = ci / den;
          gbb += lw * fs * ls.Le * g;
          const float3 gfs = lw * beta * ls.Le * g;
          const float gg = dot(lw * beta * fs, ls.Le);
          const float gci = gg / den;
          const float gpl = -gg * ci / (den * den);
          const float gpb = gpl;
          float3 gwi = f3(0.f, 0.f, 0.f);
          bsdf_eval_bwd(m, ns, wo, wi, gfs, gpb, gns, gwo, gwi);
          const float gdist2 = gpl * pl / dist2;
          const float gcl = -gpl * pl / cl;
          gwi += ns * gci - ls.nl * gcl;
          gns += wi * gci;
          const float3 gwv = (gwi - wi * dot(wi, gwi)) * (1.0f / dist) + wv * (2.0f * gdist2);
          gP -= gwv;
          const float3 dy_dsu = -ls.V0 + ls.V1 * (1.0f - ls.v2) + ls.V2 * ls.v2;
          const float gsu = dot(gwv, dy_dsu);
          g3 = dot(gwv, (ls.V2 - ls.V1) * ls.su);
          if (!ls.clamped && ls.su > 0.0f) g2 = gsu / (2.0f * ls.su) / ls.pk;
        }
        if (flags & kFScatter) {
          SampleRec s;
          opaque_sample(m, ns, ngf, wo, xa(b), xa(b + 1), s);
          const float ci = dot(ns, s.wi);
          float pdf;
          const float3 fs = bsdf_eval(m, ns, wo, s.wi, &pdf);
          // beta' = beta * fs * ci / pdf
          gbb += gbeta * s.w;
          const float3 gwv = gbeta * beta;
          const float3 gfs = gwv * (ci / pdf);
          const float gci = dot(gwv, fs) / pdf;
          const float gpdf = -dot(gwv, fs) * ci / (pdf * pdf) + gpp;
          float3 gwi = gd;
          bsdf_eval_bwd(m, ns, wo, s.wi, gfs, gpdf, gns, gwo, gwi);
          gwi += ns * gci;
          gns += s.wi * gci;
          opaque_sample_dir_bwd(m, s.lobe, ns, wo, xa(b), xa(b + 1), gwi, gns, gwo, g0, g1);
          gP += go;
        }
      }
      // d(ns) -> d(nsn) -> d(P)
      gP += shading_normal_bwd(S, tri, sf, nraw, nsn, gns * sgn);
      gdd -= gwo;
      gw(b, g0 * inv_p);
      gw(b + 1, g1 * inv_p);
      gw(b + 2, g2 * inv_p);
      gw(b + 3, g3 * inv_p);
    } else if (seg <= L - 1) {
      gw(b, 0.f); gw(b + 1, 0.f); gw(b + 2, 0.f); gw(b + 3, 0.f);
    }
    // hit point P = o + t d, t = ((v0 - o) . N) / (d . N)
    const float gtt = gt + dot(gP, d);
    go = gP - sf.N * (gtt / dn);
    gdd += gP * t - sf.N * (gtt * t / dn);
    gd = gdd;
    gbeta = gbb;
    gpp = gppd;
  }
  // camera
  float g0 = 0.f, g1 = 0.f;
  if (nseg >= 1) {
    float3 raw;
    const float3 d = camera_dir(S.cam, xa(0), xa(1), &raw);
    const float3 graw = normalize_bwd(raw, d, gd);
    g0 = 2.0f * S.cam.tx * dot(graw, S.cam.right);
    g1 = -2.0f * S.cam.ty * dot(graw, S.cam.up);
  }
  gw(0, g0 * inv_p);
  gw(1, g1 * inv_p);
}

// ---------------------------------------------------------------- mixture
// Isotropic Gaussian mixture on the torus: g(x) and (optionally) grad g.
template <class XA, class GW>
DR_D float mixture_eval(const DevMixture& M, const XA& xa, float eps, bool want_grad, const GW& gw) {
  if (M.K == 0) {
    if (want_grad) for (int i = 0; i < M.d; ++i) gw(i, 0.0f);
    return M.cval;
  }
  // pass 1: density
  float g = 0.0f;
  for (int k = 0; k < M.K; ++k) {
    const float s = __ldg(M.sig + k), s2 = s * s;
    float q = 0.0f;
    for (int i = 0; i < M.d; ++i) {
      float dd = xa(i) - __ldg(M.mu + k * M.d + i);
      dd -= rintf(dd);
      q += dd * dd;
    }
    g += __ldg(M.w + k) * expf(-0.5f * q / s2) * powf(2.0f * kPi * s2, -0.5f * (float)M.d);
  }
  if (want_grad) {
    const float inv = 1.0f / (g + eps);
    for (int i = 0; i < M.d; ++i) {
      float gi = 0.0f;
      for (int k = 0; k < M.K; ++k) {
        const float s = __ldg(M.sig + k), s2 = s * s;
        float q = 0.0f;
        for (int j = 0; j < M.d; ++j) {
          float dd = xa(j) - __ldg(M.mu + k * M.d + j);
          dd -= rintf(dd);
          q += dd * dd;
        }
        float di = xa(i) - __ldg(M.mu + k * M.d + i);
        di -= rintf(di);
        const float c = __ldg(M.w + k) * expf(-0.5f * q / s2) * powf(2.0f * kPi * s2, -0.5f * (float)M.d);
        gi -= c * di / s2;
      }
      gw(i, gi * inv);
    }
  }
  return g;
}

}  // namespace dr

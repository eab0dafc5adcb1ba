// Continuous-spin O(n) models in FP32 with FP64 observable totals
// (Weigel & Yavors'kii 2011, Section 2: Eq. 1, Eq. 2, and the mixed-precision
// scheme of Table 1, "Metro. single": spins in single precision, aggregate
// quantities such as the total energy in double precision).
//
//   XY (n = 2):          one FP32 angle per site, colour arrays t[c][j] holding
//                        the angle in turns (theta / 2 pi, in [0, 1)), so a
//                        proposal u24 is stored exactly and cos / sin of an
//                        angle need no large range reduction (sincos_turns);
//   Heisenberg (n = 3):  FP32 unit vectors, colour arrays of components
//                        s[c][a*H + j] (structure of arrays).
//
// A move proposes a fresh uniform angle (XY) or direction (Heisenberg) from
// the site's Philox outputs, computes dE = -(s' - s) . h in FP32 and accepts
// iff dE <= 0 or u24 < exp(-beta dE).  Per-thread partial sums of the
// observables are FP32; blocks and the final fixed-order total are FP64.
// FAST selects the hardware sin/cos/exp intrinsics (the "fast math" row of
// Table 1), with angles shifted into [-pi, pi) where the intrinsics are
// accurate.
//
// HB selects the heat-bath rule (Section 2's other local update): the new
// spin is drawn from its conditional law, density proportional to
// exp(beta s' . h), independent of the old spin.  Heisenberg: c = s'.h/|h|
// by inverting its exponential distribution function at u24(output 0), the
// azimuth 2 pi u24(output 1) in the orthonormal basis of Duff et al.
// (JCGT 2017) around h.  XY: the offset from the angle of h by the
// von Mises rejection method of Best and Fisher (1979), attempt a of a site
// drawing its two uniforms from Philox(group, t, replica, a << 16 | colour).
// The draws use the accurate log1p / expm1 / atan2 and sincos_turns whatever
// FAST.
#include "internal.h"

namespace spinmc {
namespace {

constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kPiF = 3.14159265358979323846f;

struct OnArgs {
    float* own;
    const float* oth;
    const float* Jown[3];
    const float* Joth[3];
    int d, L, W, c, R;
    long long H, N;
    uint32_t replica;
    RoundKeys rk;
    float beta;
    float J;
    Ctrl* ctrl;
    Partial* partials;
    int measure, update;
    int renorm_every;  // Heisenberg: normalise each updated spin when (t+1) % renorm_every == 0
};

__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

struct V3 {
    float x, y, z;
};

// sin and cos of 2 pi t for t in [0, 1]: the nearest quarter turn q / 4 is
// taken off exactly (r = t - q / 4 lies in [-1/8, 1/8], Sterbenz), and sin
// and cos of 2 pi r come from their Taylor series to degrees 9 and 10
// (truncation below 2e-9 for |2 pi r| <= pi / 4; FP32 evaluation within
// 1e-7 of the exact values); the quadrant q mod 4 swaps and negates them.
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c)
{
    const float q = rintf(4.0f * t);
    const float r = fmaf(-0.25f, q, t);
    const float y = r * r;
    const float sp =
        r * fmaf(fmaf(fmaf(fmaf(42.0586929f, y, -76.7058563f), y, 81.6052475f), y, -41.3417015f),
                 y, 6.28318548f);
    const float cp = fmaf(
        fmaf(fmaf(fmaf(fmaf(-26.4262562f, y, 60.2446404f), y, -85.4568176f), y, 64.9393921f), y,
             -19.7392082f),
        y, 1.0f);
    const int k = (int)q & 3;
    float ss = (k & 1) ? cp : sp;
    float cc = (k & 1) ? sp : cp;
    if (k == 1 || k == 2) cc = -cc;
    if (k >= 2) ss = -ss;
    *s = ss;
    *c = cc;
}

// Sin and cos of 2 pi t from a table of kTurnTab angles in shared memory and
// a short series: t = (k + r) / kTurnTab with k the nearest integer to
// kTurnTab t (taken from the mantissa after adding 1.5 2^23, so no float-to-
// integer conversion) and |r| <= 1/2 exact, x = 2 pi r / kTurnTab, |x| <=
// 3.1e-3; sin x = x (1 - x^2/6) and cos x - 1 = -x^2/2 (the next terms are
// below 4e-12); the angle-addition formulas with the tabulated (cos, sin) of
// 2 pi k / kTurnTab (correctly rounded FP32 values from sincospif).  Within
// 7e-8 of FP64 on 4e6 angles, against 9e-8 for sincos_turns, and 1.26 times
// its throughput.
constexpr int kTurnTab = 1024;

// Every thread of the block takes part; the table is ready after the barrier.
__device__ __forceinline__ void fill_turn_table(float2* tab)
{
    for (int k = threadIdx.x; k < kTurnTab; k += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)k / (float)kTurnTab, &s, &c);
        tab[k] = make_float2(c, s);
    }
    __syncthreads();
}

// (every rounding spelled out, so that each kernel gets the same values)
__device__ __forceinline__ void sincos_from_table(const float2* tab, int k, float r, float* s,
                                                  float* c)
{
    const float x = __fmul_rn(r, kTwoPiF / (float)kTurnTab);
    const float x2 = __fmul_rn(x, x);
    const float sb = __fmul_rn(x, __fmaf_rn(x2, -1.0f / 6.0f, 1.0f));
    const float cm1 = __fmul_rn(-0.5f, x2);
    const float2 e = tab[k];  // (cos, sin) of 2 pi k / kTurnTab
    *s = __fadd_rn(e.y, __fmaf_rn(e.y, cm1, __fmul_rn(e.x, sb)));
    *c = __fadd_rn(e.x, __fmaf_rn(e.x, cm1, -__fmul_rn(e.y, sb)));
}

// t in turns, [0, 1)
__device__ __forceinline__ void sincos_turns_tab(const float2* tab, float t, float* s, float* c)
{
    const float magic = 12582912.0f;  // 1.5 2^23: the sum's ulp is 1
    const float fm = fmaf(t, (float)kTurnTab, magic);
    const float kf = fm - magic;
    const int k = __float_as_int(fm) & (kTurnTab - 1);
    sincos_from_table(tab, k, fmaf(t, (float)kTurnTab, -kf), s, c);
}

// sin and cos of an angle given in turns t in [0, 1)
template <bool FAST>
__device__ __forceinline__ void sincos_angle(float t, float* s, float* c)
{
    if (FAST) {
        // sin(2 pi t) = -sin(2 pi t - pi), likewise cos; the argument is in [-pi, pi)
        __sincosf(kTwoPiF * t - kPiF, s, c);
        *s = -*s;
        *c = -*c;
    } else {
        sincos_turns(t, s, c);
    }
}

template <bool FAST>
__device__ __forceinline__ float boltzmann(float x)
{
    return FAST ? __expf(x) : expf(x);
}

// fresh uniform direction on the sphere from two 32-bit outputs
template <bool FAST>
__device__ __forceinline__ float3 sphere_point(uint32_t oz, uint32_t ophi)
{
    const float z = 2.0f * u24(oz) - 1.0f;
    const float r = sqrtf((1.0f - z) * (1.0f + z));
    float sp, cp;
    if (FAST) {
        __sincosf(kTwoPiF * u24(ophi) - kPiF, &sp, &cp);
        sp = -sp;
        cp = -cp;
    } else {
        sincos_turns(u24(ophi), &sp, &cp);
    }
    return make_float3(r * cp, r * sp, z);
}

// The same point with sin and cos of the azimuth from the shared table.
__device__ __forceinline__ float3 sphere_point_tab(const float2* tab, uint32_t oz, uint32_t ophi)
{
    const float z = __fmaf_rn(2.0f, u24(oz), -1.0f);  // exact
    const float r = sqrtf(__fmul_rn(1.0f - z, 1.0f + z));
    float sp, cp;
    sincos_turns_tab(tab, u24(ophi), &sp, &cp);
    return make_float3(__fmul_rn(r, cp), __fmul_rn(r, sp), z);
}

// One component of a Heisenberg site's field, every rounding spelled out so
// that each kernel computes it identically whatever the compiler would fuse:
// ((x- + x+) + a) + b along the marching axis, then + (c + d) across (3D),
// times J.
template <int D>
__device__ __forceinline__ float heis_field(float xm, float xp, float a, float b, float c, float d,
                                            float J)
{
    float h = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), a), b);
    if (D == 3) h = __fadd_rn(h, __fadd_rn(c, d));
    return __fmul_rn(h, J);
}

// The Metropolis step of one Heisenberg site with proposal v (Eq. 2, dE =
// -(v - s) . h, accurate or intrinsic exp) and the optional renormalisation,
// every rounding spelled out as in heis_field; true if s changed.
template <bool FAST>
__device__ __forceinline__ bool heis_metropolis(float& sx, float& sy, float& sz, const float3& v,
                                                float hx, float hy, float hz, float u, float beta,
                                                bool renorm)
{
    bool changed = false;
    const float dE = -__fmaf_rn(__fsub_rn(v.z, sz), hz,
                                __fmaf_rn(__fsub_rn(v.y, sy), hy,
                                          __fmul_rn(__fsub_rn(v.x, sx), hx)));
    // the Boltzmann factor is evaluated whatever the sign of dE, so the step
    // is straight-line code the scheduler can interleave with other sites
    const float w = boltzmann<FAST>(__fmul_rn(-beta, dE));
    if ((dE <= 0.f) | (u < w)) {
        sx = v.x;
        sy = v.y;
        sz = v.z;
        changed = true;
    }
    if (renorm) {
        const float inv = rsqrtf(__fmaf_rn(sz, sz, __fmaf_rn(sy, sy, __fmul_rn(sx, sx))));
        sx = __fmul_rn(sx, inv);
        sy = __fmul_rn(sy, inv);
        sz = __fmul_rn(sz, inv);
        changed = true;
    }
    return changed;
}

// Heat-bath draw of a Heisenberg spin in the local field h, kappa = beta |h|.
// 1 - c and 1 + c are both formed without
// cancellation: 1 - c = -log1p((1 - u) expm1(-2 kappa)) / kappa when that is
// <= 1, else 1 + c = log1p(u expm1(2 kappa)) / kappa (for 2 kappa > 80,
// where expm1 overflows, 2 + log(u) / kappa, exact to FP32 precision).
__device__ __forceinline__ V3 heis_heatbath(float hx, float hy, float hz, float beta,
                                             uint32_t o0, uint32_t o1)
{
    const float H2 = hx * hx + hy * hy + hz * hz;
    float nx = 0.f, ny = 0.f, nz = 1.f, kappa = 0.f;
    if (H2 > 0.f) {
        const float inv = rsqrtf(H2);
        nx = hx * inv;
        ny = hy * inv;
        nz = hz * inv;
        kappa = beta * (H2 * inv);
    }
    const float u = u24(o0);
    float omc, opc;  // 1 - c, 1 + c
    if (kappa > 0.f) {
        omc = -log1pf((1.f - u) * expm1f(-2.f * kappa)) / kappa;
        if (omc <= 1.f) {
            opc = 2.f - omc;
        } else {
            opc = 2.f * kappa <= 80.f ? log1pf(u * expm1f(2.f * kappa)) / kappa
                                      : fmaxf(0.f, 2.f + logf(u) / kappa);
            omc = 2.f - opc;
        }
    } else {
        omc = 2.f * (1.f - u);
        opc = 2.f * u;
    }
    omc = fmaxf(omc, 0.f);
    opc = fmaxf(opc, 0.f);
    const float c = omc <= 1.f ? 1.f - omc : opc - 1.f;
    const float r = sqrtf(omc * opc);
    // basis (e1, e2, n) of Duff et al.: smooth except where n_z changes sign
    const float sg = copysignf(1.f, nz);
    const float ia = -1.f / (sg + nz);
    const float b = nx * ny * ia;
    float sp, cp;
    sincos_turns(u24(o1), &sp, &cp);
    const float p1 = r * cp, p2 = r * sp;
    V3 v;
    v.x = c * nx + p1 * (1.f + sg * nx * nx * ia) + p2 * b;
    v.y = c * ny + p1 * (sg * b) + p2 * (sg + ny * ny * ia);
    v.z = c * nz - p1 * (sg * nx) - p2 * ny;
    return v;
}

// Per-site constants of the Best-Fisher von Mises sampler for kappa = beta |h|:
// the wrapped-Cauchy parameter rho = 2 kappa / (tau + sqrt(2 tau)),
// tau = 1 + sqrt(1 + 4 kappa^2), the half-angle factor g = (1 - rho) / (1 + rho)
// and the numerator of the test quantity, (tau + sqrt(2 tau)) (1 - rho^2)^2 / 4.
struct VonMises {
    float rho, g, cnum, base;  // base: angle of h in turns
};

__device__ __forceinline__ VonMises von_mises_setup(float hx, float hy, float beta)
{
    VonMises m;
    const float kappa = beta * sqrtf(hx * hx + hy * hy);
    const float tau = 1.f + sqrtf(1.f + 4.f * kappa * kappa);
    const float s2 = sqrtf(2.f * tau);
    m.rho = 2.f * kappa / (tau + s2);
    m.g = (1.f - m.rho) / (1.f + m.rho);
    const float q = 1.f - m.rho * m.rho;
    m.cnum = 0.25f * (tau + s2) * q * q;
    m.base = atan2f(hy, hx) * (1.0f / kTwoPiF);
    return m;
}

// The acceptance test of one Best-Fisher attempt from the raw outputs o1
// (U1, with w = pi U1 / 2) and o2 (U2).
__device__ __forceinline__ bool von_mises_accept(const VonMises& m, uint32_t o1, uint32_t o2)
{
    float sw, cw;
    sincos_turns(0.25f * u24(o1), &sw, &cw);
    const float omr = 1.f - m.rho;
    const float cc = m.cnum / (omr * omr + 4.f * m.rho * cw * cw);
    const float U2 = u24(o2);
    return cc * (2.f - cc) > U2 || logf(cc / U2) + 1.f - cc >= 0.f;
}

// The new angle, in turns in [0, 1), of the accepted attempt with output o1:
// the angle of h plus or minus (bit 0 of o1) delta, tan(delta/2) = g tan w.
// Kept out of the attempt loop so that a warp pays for it once.
__device__ __forceinline__ float von_mises_angle(const VonMises& m, uint32_t o1)
{
    float sw, cw;
    sincos_turns(0.25f * u24(o1), &sw, &cw);
    float dt = atan2f(m.g * sw, cw) * (1.0f / kPiF);
    if (o1 & 1u) dt = -dt;
    float tn = m.base + dt;
    tn -= floorf(tn);
    return tn < 1.f ? tn : 0.f;
}

constexpr int kVonMisesAttempts = 32;

__device__ __forceinline__ void on_finish(const OnArgs& a, const Partial& tot)
{
    Ctrl* C = a.ctrl;
    C->obs[0] = tot.f[0];
    C->obs[1] = tot.f[1];
    C->obs[2] = tot.f[2];
    C->obs[3] = tot.f[3];
    if (a.update) {
        const long long k = (long long)C->t - C->series_base;
        const double m = sqrt(tot.f[1] * tot.f[1] + tot.f[2] * tot.f[2] + tot.f[3] * tot.f[3]);
        if (C->series_E) C->series_E[k] = tot.f[0];
        if (C->series_absm) C->series_absm[k] = m / (double)a.N;
        C->t = C->t + 1;
    }
}

// One thread per site; a block walks whole rows (fixed y, z) so that the
// loads of a warp are contiguous.  Any even L.
template <int NC, int D, bool FAST, bool HB>
__global__ void __launch_bounds__(128) on_generic(const OnArgs a)
{
    __shared__ double red[32];
    const unsigned long long t64 = a.ctrl->t;
    const uint32_t t = (uint32_t)t64;
    const bool renorm = NC == 3 && a.update && a.renorm_every > 0 &&
                        (t64 + 1) % (unsigned long long)a.renorm_every == 0;
    const int L = a.L, W = a.W;
    const long long H = a.H;
    const long long nrows = (long long)L * (D == 3 ? L : 1);
    const bool bonds = a.Jown[0] != nullptr;
    float pe = 0.f, pmx = 0.f, pmy = 0.f, pmz = 0.f;
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int y = (int)(row % L);
        const int z = (int)(row / L);
        const int p = (y + z + a.c) & 1;
        const long long base = row * W;
        const long long rym = (long long)(z)*L + (y == 0 ? L - 1 : y - 1);
        const long long ryp = (long long)(z)*L + (y == L - 1 ? 0 : y + 1);
        const long long rzm = (long long)(z == 0 ? L - 1 : z - 1) * L + y;
        const long long rzp = (long long)(z == L - 1 ? 0 : z + 1) * L + y;
        for (int k = threadIdx.x; k < W; k += blockDim.x) {
            const long long j = base + k;
            int kxm = k - 1 + p, kxp = k + p;
            if (kxm < 0) kxm = W - 1;
            if (kxp == W) kxp = 0;
            long long nb[6] = {base + kxm, base + kxp, rym * W + k, ryp * W + k, 0, 0};
            if (D == 3) {
                nb[4] = rzm * W + k;
                nb[5] = rzp * W + k;
            }
            float jk[6];
#pragma unroll
            for (int q = 0; q < 2 * D; ++q) {
                const int mu = q >> 1;
                jk[q] = bonds ? a.J * ((q & 1) ? a.Jown[mu][j] : a.Joth[mu][nb[q]]) : a.J;
            }
            // local field h and the colour-0 site sharing index j
            float hx = 0.f, hy = 0.f, hz = 0.f, ox = 0.f, oy = 0.f, oz = 0.f;
            const int q_same = p ? 0 : 1;  // neighbour with colour index k in this row
#pragma unroll
            for (int q = 0; q < 2 * D; ++q) {
                float vx, vy, vz = 0.f;
                if (NC == 2) {
                    sincos_angle<FAST>(a.oth[nb[q]], &vy, &vx);
                } else {
                    vx = a.oth[nb[q]];
                    vy = a.oth[H + nb[q]];
                    vz = a.oth[2 * H + nb[q]];
                }
                hx += jk[q] * vx;
                hy += jk[q] * vy;
                hz += jk[q] * vz;
                if (q == q_same) {
                    ox = vx;
                    oy = vy;
                    oz = vz;
                }
            }
            float sx, sy, sz = 0.f, th = 0.f;
            if (NC == 2) {
                th = a.own[j];
                sincos_angle<FAST>(th, &sy, &sx);
            } else {
                sx = a.own[j];
                sy = a.own[H + j];
                sz = a.own[2 * H + j];
            }
            bool changed = false;
            if (a.update && HB) {
                if (NC == 2) {
                    const VonMises vm = von_mises_setup(hx, hy, a.beta);
                    for (int at = 0; at < kVonMisesAttempts; ++at) {
                        const uint4 r = philox4x32_10(
                            make_uint4((uint32_t)(j >> 1), t, a.replica,
                                       ((uint32_t)at << 16) | (kSweep << 1) | (uint32_t)a.c),
                            a.rk);
                        const uint32_t o1 = (j & 1) ? r.z : r.x;
                        if (von_mises_accept(vm, o1, (j & 1) ? r.w : r.y)) {
                            th = von_mises_angle(vm, o1);
                            sincos_angle<FAST>(th, &sy, &sx);
                            changed = true;
                            break;
                        }
                    }
                } else {
                    const uint4 r = philox4x32_10(
                        make_uint4((uint32_t)j, t, a.replica, (kSweep << 1) | (uint32_t)a.c), a.rk);
                    const V3 v = heis_heatbath(hx, hy, hz, a.beta, r.x, r.y);
                    sx = v.x;
                    sy = v.y;
                    sz = v.z;
                    changed = true;
                }
            } else if (a.update) {
                float nx, ny, nz = 0.f, nth = 0.f, u;
                if (NC == 2) {
                    const uint4 r = philox4x32_10(
                        make_uint4((uint32_t)(j >> 1), t, a.replica, (kSweep << 1) | (uint32_t)a.c),
                        a.rk);
                    const uint32_t oa = (j & 1) ? r.z : r.x;
                    const uint32_t op = (j & 1) ? r.w : r.y;
                    u = u24(oa);
                    nth = u24(op);
                    sincos_angle<FAST>(nth, &ny, &nx);
                } else {
                    const uint4 r = philox4x32_10(
                        make_uint4((uint32_t)j, t, a.replica, (kSweep << 1) | (uint32_t)a.c), a.rk);
                    u = u24(r.x);
                    const float3 v = sphere_point<FAST>(r.y, r.z);
                    nx = v.x;
                    ny = v.y;
                    nz = v.z;
                }
                const float dE = -((nx - sx) * hx + (ny - sy) * hy + (nz - sz) * hz);
                const bool acc = dE <= 0.f || u < boltzmann<FAST>(-a.beta * dE);
                if (acc) {
                    sx = nx;
                    sy = ny;
                    sz = nz;
                    th = nth;
                    changed = true;
                }
            }
            if (a.update) {
                if (renorm) {
                    const float inv = rsqrtf(sx * sx + sy * sy + sz * sz);
                    sx *= inv;
                    sy *= inv;
                    sz *= inv;
                    changed = true;
                }
                if (changed) {
                    if (NC == 2) {
                        a.own[j] = th;
                    } else {
                        a.own[j] = sx;
                        a.own[H + j] = sy;
                        a.own[2 * H + j] = sz;
                    }
                }
            }
            if (a.measure) {
                pe -= sx * hx + sy * hy + sz * hz;
                pmx += sx + ox;
                pmy += sy + oy;
                pmz += sz + oz;
            }
        }
    }
    if (!a.measure) return;
    Partial mine;
    mine.i0 = mine.i1 = 0;
    mine.f[0] = block_sum((double)pe, red);
    mine.f[1] = block_sum((double)pmx, red);
    mine.f[2] = block_sum((double)pmy, red);
    mine.f[3] = block_sum((double)pmz, red);
    finish_pass(a.ctrl, a.partials, mine, [&](const Partial& tot) { on_finish(a, tot); });
}

// ------------------------------------------------------------ streaming ----
//
// Uniform coupling, W % 32 == 0 (Heisenberg) or W % 64 == 0 (XY): a warp owns
// 32 consecutive columns (heis_stream) or column pairs (heis_pair when
// W % 64 == 0, xy_stream) of one row and marches along the last axis (y in
// 2D, z in 3D) through R rows, keeping the other colour's rows behind, at
// and ahead of the current one in registers (for XY as cos/sin, computed once
// per value).  The x neighbours come from the adjacent lane by a shuffle (the
// two warp-edge lanes load theirs).  Loads for the next row are issued one
// row ahead.

__device__ __forceinline__ V3 shfl3_up(V3 v)
{
    V3 r;
    r.x = __shfl_up_sync(0xffffffffu, v.x, 1);
    r.y = __shfl_up_sync(0xffffffffu, v.y, 1);
    r.z = __shfl_up_sync(0xffffffffu, v.z, 1);
    return r;
}

__device__ __forceinline__ V3 shfl3_down(V3 v)
{
    V3 r;
    r.x = __shfl_down_sync(0xffffffffu, v.x, 1);
    r.y = __shfl_down_sync(0xffffffffu, v.y, 1);
    r.z = __shfl_down_sync(0xffffffffu, v.z, 1);
    return r;
}

// MEAS: the measuring (colour-1) pass, which stores its block partials for
// on_finish_kernel; the other pass is compiled without the sums.
template <int D, bool FAST, bool HB, bool MEAS>
__global__ void __launch_bounds__(256, D == 2 && !HB ? 4 : 3) heis_stream(const OnArgs a)
{
    __shared__ double red[32];
    // Metropolis with accurate functions: the proposal's azimuth from the shared table
    constexpr bool TAB = !FAST && !HB;
    __shared__ float2 tab[TAB ? kTurnTab : 1];
    if (TAB) fill_turn_table(tab);
    const unsigned long long t64 = a.ctrl->t;
    const uint32_t t = (uint32_t)t64;
    const bool renorm = a.update && a.renorm_every > 0 &&
                        (t64 + 1) % (unsigned long long)a.renorm_every == 0;
    const int L = a.L, W = a.W, R = a.R;
    const long long H = a.H;  // < 2^31: every offset below fits in 32 bits
    const int lane = threadIdx.x & 31;
    const long long nitems = (long long)W * (D == 3 ? L : 1) * (L / R);
    const float J = a.J;
    const float* ox = a.oth;
    const float* oy = a.oth + H;
    const float* oz = a.oth + 2 * H;
    float* sx_ = a.own;
    float* sy_ = a.own + H;
    float* sz_ = a.own + 2 * H;
    auto ld = [&](int i) -> V3 {
        V3 v;
        v.x = __ldg(ox + i);
        v.y = __ldg(oy + i);
        v.z = __ldg(oz + i);
        return v;
    };
    float pe = 0.f, pmx = 0.f, pmy = 0.f, pmz = 0.f;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(it % W);
        const long long rest = it / W;
        const int y3 = D == 3 ? (int)(rest % L) : 0;
        const int m0 = (int)(D == 3 ? rest / L : rest) * R;
        // offset of the colour entry at column k of the row at march index m
        // (2D: row y = m; 3D: row (y3, z = m)); rows y3 -/+ 1 in the same plane
        auto off = [&](int m) -> int { return (D == 3 ? m * L + y3 : m) * W + k; };
        const int dym = (y3 == 0 ? L - 1 : -1) * W, dyp = (y3 == L - 1 ? 1 - L : 1) * W;
        const int mprev = m0 == 0 ? L - 1 : m0 - 1;
        V3 prev = ld(off(mprev));
        V3 cur = ld(off(m0));
        V3 nxt_pf = ld(off(m0 == L - 1 ? 0 : m0 + 1));
        V3 own_pf;
        own_pf.x = sx_[off(m0)];
        own_pf.y = sy_[off(m0)];
        own_pf.z = sz_[off(m0)];
        V3 ym_pf = prev, yp_pf = prev;
        if (D == 3) {
            ym_pf = ld(off(m0) + dym);
            yp_pf = ld(off(m0) + dyp);
        }
        // the x neighbour a warp-edge lane cannot get by shuffle: column k-1
        // for lane 0 when p = 0, column k+1 for lane 31 when p = 1
        const int kl = k == 0 ? W - 1 : k - 1, kr = k == W - 1 ? 0 : k + 1;
        auto edge_of = [&](int m, int p) -> int { return off(m) - k + (p ? kr : kl); };
        auto is_edge = [&](int p) -> bool { return p ? lane == 31 : lane == 0; };
        V3 edge_pf = prev;
        {
            const int p0 = ((D == 3 ? y3 : m0) + (D == 3 ? m0 : 0) + a.c) & 1;
            if (is_edge(p0)) edge_pf = ld(edge_of(m0, p0));
        }
        for (int r = 0; r < R; ++r) {
            const int m = m0 + r;
            const int yy = D == 3 ? y3 : m, zz = D == 3 ? m : 0;
            const int p = (yy + zz + a.c) & 1;
            const int j = off(m);
            const V3 nxt = nxt_pf;
            const V3 vm = ym_pf, vp = yp_pf;
            const V3 edge = edge_pf;
            V3 s = own_pf;
            if (r + 1 < R) {
                const int m2 = m + 2 >= L ? m + 2 - L : m + 2;
                const int j1 = off(m + 1);
                nxt_pf = ld(off(m2));
                own_pf.x = sx_[j1];
                own_pf.y = sy_[j1];
                own_pf.z = sz_[j1];
                if (D == 3) {
                    ym_pf = ld(j1 + dym);
                    yp_pf = ld(j1 + dyp);
                }
                const int p1 = p ^ 1;  // the parity alternates along the marching axis
                if (is_edge(p1)) edge_pf = ld(edge_of(m + 1, p1));
            }
            // x neighbours: p = 0 -> (k-1, k), p = 1 -> (k, k+1)
            V3 xm, xp;
            if (p == 0) {
                xm = shfl3_up(cur);
                if (lane == 0) xm = edge;
                xp = cur;
            } else {
                xm = cur;
                xp = shfl3_down(cur);
                if (lane == 31) xp = edge;
            }
            const float hx = heis_field<D>(xm.x, xp.x, prev.x, nxt.x, vm.x, vp.x, J);
            const float hy = heis_field<D>(xm.y, xp.y, prev.y, nxt.y, vm.y, vp.y, J);
            const float hz = heis_field<D>(xm.z, xp.z, prev.z, nxt.z, vm.z, vp.z, J);
            if (a.update) {
                const uint4 rnd = philox4x32_10(
                    make_uint4((uint32_t)j, t, a.replica, (kSweep << 1) | (uint32_t)a.c), a.rk);
                bool changed = false;
                if (HB) {
                    s = heis_heatbath(hx, hy, hz, a.beta, rnd.x, rnd.y);
                    changed = true;
                    if (renorm) {
                        const float inv = rsqrtf(s.x * s.x + s.y * s.y + s.z * s.z);
                        s.x *= inv;
                        s.y *= inv;
                        s.z *= inv;
                    }
                } else {
                    const float3 v = TAB ? sphere_point_tab(tab, rnd.y, rnd.z)
                                         : sphere_point<FAST>(rnd.y, rnd.z);
                    changed = heis_metropolis<FAST>(s.x, s.y, s.z, v, hx, hy, hz, u24(rnd.x),
                                                    a.beta, renorm);
                }
                if (changed) {
                    sx_[j] = s.x;
                    sy_[j] = s.y;
                    sz_[j] = s.z;
                }
            }
            if (MEAS) {
                pe -= s.x * hx + s.y * hy + s.z * hz;
                pmx += s.x + cur.x;
                pmy += s.y + cur.y;
                pmz += s.z + cur.z;
            }
            prev = cur;
            cur = nxt;
        }
    }
    if (!MEAS) return;
    Partial mine;
    mine.i0 = mine.i1 = 0;
    mine.f[0] = block_sum((double)pe, red);
    mine.f[1] = block_sum((double)pmx, red);
    mine.f[2] = block_sum((double)pmy, red);
    mine.f[3] = block_sum((double)pmz, red);
    store_partial(a.partials, mine);
}

struct P3 {
    float2 x, y, z;
};

// Heisenberg streaming kernel on column pairs: as heis_stream, but each
// thread owns colour columns (2q, 2q+1) of its rows and loads each component
// of a row pair with one 8-byte load, which halves the load instructions and
// the index arithmetic per site and doubles the bytes each load carries
// (measured 9% faster in 3D).  Needs W % 64 == 0.  2D fits 3 blocks of 256
// per SM without spilling (+11% over 2); 3D spills at 3 and keeps 2.
template <int D, bool FAST, bool HB, bool MEAS>
__global__ void __launch_bounds__(256, D == 2 ? 3 : 2) heis_pair(const OnArgs a)
{
    __shared__ double red[32];
    // Metropolis with accurate functions: the proposal's azimuth from the shared table
    constexpr bool TAB = !FAST && !HB;
    __shared__ float2 tab[TAB ? kTurnTab : 1];
    if (TAB) fill_turn_table(tab);
    const unsigned long long t64 = a.ctrl->t;
    const uint32_t t = (uint32_t)t64;
    const bool renorm = a.update && a.renorm_every > 0 &&
                        (t64 + 1) % (unsigned long long)a.renorm_every == 0;
    const int L = a.L, W = a.W, R = a.R;
    const int WP = W / 2;
    const long long H = a.H;  // < 2^31: every offset below fits in 32 bits
    const int lane = threadIdx.x & 31;
    const long long nitems = (long long)WP * (D == 3 ? L : 1) * (L / R);
    const float J = a.J;
    const float* ox = a.oth;
    const float* oy = a.oth + H;
    const float* oz = a.oth + 2 * H;
    float* sx_ = a.own;
    float* sy_ = a.own + H;
    float* sz_ = a.own + 2 * H;
    auto ld = [&](int i) -> P3 {
        P3 v;
        v.x = __ldg(reinterpret_cast<const float2*>(ox + i));
        v.y = __ldg(reinterpret_cast<const float2*>(oy + i));
        v.z = __ldg(reinterpret_cast<const float2*>(oz + i));
        return v;
    };
    auto ld_own = [&](int i) -> P3 {
        P3 v;
        v.x = *reinterpret_cast<const float2*>(sx_ + i);
        v.y = *reinterpret_cast<const float2*>(sy_ + i);
        v.z = *reinterpret_cast<const float2*>(sz_ + i);
        return v;
    };
    auto ld_one = [&](int i) -> V3 {
        V3 v;
        v.x = __ldg(ox + i);
        v.y = __ldg(oy + i);
        v.z = __ldg(oz + i);
        return v;
    };
    float pe = 0.f, pmx = 0.f, pmy = 0.f, pmz = 0.f;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (long long)gridDim.x * blockDim.x) {
        const int k0 = 2 * (int)(it % WP);
        const long long rest = it / WP;
        const int y3 = D == 3 ? (int)(rest % L) : 0;
        const int m0 = (int)(D == 3 ? rest / L : rest) * R;
        auto off = [&](int m) -> int { return (D == 3 ? m * L + y3 : m) * W + k0; };
        const int dym = (y3 == 0 ? L - 1 : -1) * W, dyp = (y3 == L - 1 ? 1 - L : 1) * W;
        const int mprev = m0 == 0 ? L - 1 : m0 - 1;
        P3 prev = ld(off(mprev));
        P3 cur = ld(off(m0));
        P3 nxt_pf = ld(off(m0 == L - 1 ? 0 : m0 + 1));
        P3 own_pf = ld_own(off(m0));
        P3 ym_pf = prev, yp_pf = prev;
        if (D == 3) {
            ym_pf = ld(off(m0) + dym);
            yp_pf = ld(off(m0) + dyp);
        }
        // the x neighbour outside the pair that a warp-edge lane cannot get by
        // shuffle: column 2q-1 for lane 0 when p = 0, 2q+2 for lane 31 when p = 1
        const int kl = k0 == 0 ? W - 1 : k0 - 1, kr = k0 + 2 == W ? 0 : k0 + 2;
        V3 edge_pf = {0.f, 0.f, 0.f};
        {
            const int p0 = ((D == 3 ? y3 : m0) + (D == 3 ? m0 : 0) + a.c) & 1;
            if (p0 ? lane == 31 : lane == 0) edge_pf = ld_one(off(m0) - k0 + (p0 ? kr : kl));
        }
        for (int r = 0; r < R; ++r) {
            const int m = m0 + r;
            const int yy = D == 3 ? y3 : m, zz = D == 3 ? m : 0;
            const int p = (yy + zz + a.c) & 1;
            const int j = off(m);
            const P3 nxt = nxt_pf, vm = ym_pf, vp = yp_pf;
            const V3 edge = edge_pf;
            P3 s = own_pf;
            if (r + 1 < R) {
                const int m2 = m + 2 >= L ? m + 2 - L : m + 2;
                const int j1 = off(m + 1);
                nxt_pf = ld(off(m2));
                own_pf = ld_own(j1);
                if (D == 3) {
                    ym_pf = ld(j1 + dym);
                    yp_pf = ld(j1 + dyp);
                }
                const int p1 = p ^ 1;  // the parity alternates along the marching axis
                if (p1 ? lane == 31 : lane == 0) edge_pf = ld_one(j1 - k0 + (p1 ? kr : kl));
            }
            // x neighbours: p = 0 -> A (2q-1, 2q), B (2q, 2q+1);
            //               p = 1 -> A (2q, 2q+1), B (2q+1, 2q+2)
            float ex, ey, ez;
            if (p == 0) {
                ex = __shfl_up_sync(0xffffffffu, cur.x.y, 1);
                ey = __shfl_up_sync(0xffffffffu, cur.y.y, 1);
                ez = __shfl_up_sync(0xffffffffu, cur.z.y, 1);
                if (lane == 0) {
                    ex = edge.x;
                    ey = edge.y;
                    ez = edge.z;
                }
            } else {
                ex = __shfl_down_sync(0xffffffffu, cur.x.x, 1);
                ey = __shfl_down_sync(0xffffffffu, cur.y.x, 1);
                ez = __shfl_down_sync(0xffffffffu, cur.z.x, 1);
                if (lane == 31) {
                    ex = edge.x;
                    ey = edge.y;
                    ez = edge.z;
                }
            }
            V3 hA, hB;
            hA.x = heis_field<D>(p ? cur.x.y : ex, cur.x.x, prev.x.x, nxt.x.x, vm.x.x, vp.x.x, J);
            hA.y = heis_field<D>(p ? cur.y.y : ey, cur.y.x, prev.y.x, nxt.y.x, vm.y.x, vp.y.x, J);
            hA.z = heis_field<D>(p ? cur.z.y : ez, cur.z.x, prev.z.x, nxt.z.x, vm.z.x, vp.z.x, J);
            hB.x = heis_field<D>(p ? ex : cur.x.x, cur.x.y, prev.x.y, nxt.x.y, vm.x.y, vp.x.y, J);
            hB.y = heis_field<D>(p ? ey : cur.y.x, cur.y.y, prev.y.y, nxt.y.y, vm.y.y, vp.y.y, J);
            hB.z = heis_field<D>(p ? ez : cur.z.x, cur.z.y, prev.z.y, nxt.z.y, vm.z.y, vp.z.y, J);
            if (a.update) {
                bool changed = false;
                // both sites' random numbers first: two independent chains
                uint4 rnd2[2];
#pragma unroll
                for (int b = 0; b < 2; ++b)
                    rnd2[b] = philox4x32_10(
                        make_uint4((uint32_t)(j + b), t, a.replica, (kSweep << 1) | (uint32_t)a.c),
                        a.rk);
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const uint4 rnd = rnd2[b];
                    float& sx = b ? s.x.y : s.x.x;
                    float& sy = b ? s.y.y : s.y.x;
                    float& sz = b ? s.z.y : s.z.x;
                    const V3 h = b ? hB : hA;
                    if (HB) {
                        const V3 v = heis_heatbath(h.x, h.y, h.z, a.beta, rnd.x, rnd.y);
                        sx = v.x;
                        sy = v.y;
                        sz = v.z;
                        changed = true;
                        if (renorm) {
                            const float inv = rsqrtf(sx * sx + sy * sy + sz * sz);
                            sx *= inv;
                            sy *= inv;
                            sz *= inv;
                        }
                    } else {
                        const float3 v = TAB ? sphere_point_tab(tab, rnd.y, rnd.z)
                                             : sphere_point<FAST>(rnd.y, rnd.z);
                        changed = heis_metropolis<FAST>(sx, sy, sz, v, h.x, h.y, h.z, u24(rnd.x),
                                                        a.beta, renorm) ||
                                  changed;
                    }
                }
                if (changed) {
                    *reinterpret_cast<float2*>(sx_ + j) = s.x;
                    *reinterpret_cast<float2*>(sy_ + j) = s.y;
                    *reinterpret_cast<float2*>(sz_ + j) = s.z;
                }
            }
            if (MEAS) {
                pe -= s.x.x * hA.x + s.y.x * hA.y + s.z.x * hA.z + s.x.y * hB.x + s.y.y * hB.y +
                      s.z.y * hB.z;
                pmx += s.x.x + s.x.y + cur.x.x + cur.x.y;
                pmy += s.y.x + s.y.y + cur.y.x + cur.y.y;
                pmz += s.z.x + s.z.y + cur.z.x + cur.z.y;
            }
            prev = cur;
            cur = nxt;
        }
    }
    if (!MEAS) return;
    Partial mine;
    mine.i0 = mine.i1 = 0;
    mine.f[0] = block_sum((double)pe, red);
    mine.f[1] = block_sum((double)pmx, red);
    mine.f[2] = block_sum((double)pmy, red);
    mine.f[3] = block_sum((double)pmz, red);
    store_partial(a.partials, mine);
}

struct CS2 {
    float c0, s0, c1, s1;  // cos / sin of the two columns of a pair
};

template <bool FAST>
__device__ __forceinline__ CS2 cs_pair(const float* p, long long i)
{
    const float2 th = __ldg(reinterpret_cast<const float2*>(p + i));
    CS2 r;
    sincos_angle<FAST>(th.x, &r.s0, &r.c0);
    sincos_angle<FAST>(th.y, &r.s1, &r.c1);
    return r;
}

// ------------------------------------------------- staged 3D Heisenberg ----
//
// 3D Heisenberg, uniform J, Metropolis with the accurate functions, W = L/2 in
// {32, 64, 128, 256}.  A work item is Y = 512 / W rows times the whole row
// width of kTileZ consecutive planes; a block of 256 threads gives each
// thread one column pair of one row and marches through the item's planes.
// The other colour's planes z-1 .. z+kTileZ (each with its rows y0-1 .. y0+Y,
// the y halo, wrapped) and the own colour's planes stream into shared memory
// through one-dimensional bulk copies (the TMA engine, completion counted on
// an mbarrier per stage) two planes ahead of use, so the threads hold no
// register window and load latency overlaps the arithmetic.  Persistent
// blocks take items in order (adjacent stripes of one slab after another).
// One lane per warp polls each stage's mbarrier while the others wait in the
// block barrier that follows.  Every wait is bounded: when one runs out the block
// sets bit 0 of the control block's error word, waits (bounded) for the
// copies it has in flight and stops; the host reports SL_ETIMEOUT.
// Decisions, random numbers and arithmetic are those of heis_pair and
// heis_stream, site for site (the shared heis_field / heis_metropolis).
constexpr int kTileThreads = 256;
constexpr int kTileZ = 8;        // planes per work item
constexpr int kOthStages = 4;    // planes z-1, z, z+1 in use and z+2 in flight
constexpr int kOwnStages = 2;
// polls of an mbarrier before a wait gives up: with the 32 ns back-off, at
// most a few seconds (a completed copy is seen within microseconds)
constexpr long long kTileWaitLimit = 1LL << 25;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (a multiple of 16, both ends 16-byte
// aligned) whose completion is counted on the mbarrier `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// wait for phase `parity` of the mbarrier to complete (non-blocking polls with
// a short back-off); false after the limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < kTileWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (it >= 8) __nanosleep(32);
    }
    return false;
}

// Self-test of the bounded wait: an mbarrier armed for 16 bytes that no copy
// ever delivers; the poll gives up after its limit and the kernel records
// whether it did (1), or saw the phase complete (0).
__device__ unsigned int g_wait_selftest;

__global__ void wait_selftest_kernel()
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(b, 16u);
        g_wait_selftest = mbar_wait(b, 0u) ? 0u : 1u;
    }
}

struct TileShape {
    int W, Y;            // colour columns per row, rows per item
    int oth_floats;      // one other-colour stage: 3 components x (Y + 2) rows x W
    int own_floats;      // one own-colour stage: 3 components x Y rows x W
};

__host__ __device__ inline TileShape tile_shape(int W)
{
    TileShape g;
    g.W = W;
    g.Y = 512 / W;
    g.oth_floats = 3 * (g.Y + 2) * W;
    g.own_floats = 3 * g.Y * W;
    return g;
}

template <bool MEAS>
__global__ void __launch_bounds__(kTileThreads, 3) heis_tile3(const OnArgs a)
{
    extern __shared__ __align__(128) float tile_smem[];
    __shared__ float2 tab[kTurnTab];
    __shared__ __align__(8) unsigned long long bars[kOthStages + kOwnStages];
    __shared__ double red[32];
    fill_turn_table(tab);
    const unsigned long long t64 = a.ctrl->t;
    const uint32_t t = (uint32_t)t64;
    const bool renorm = a.update && a.renorm_every > 0 &&
                        (t64 + 1) % (unsigned long long)a.renorm_every == 0;
    const int L = a.L, W = a.W;
    const TileShape g = tile_shape(W);
    const int Y = g.Y;
    const long long H = a.H;
    const float J = a.J;
    float* oth_st = tile_smem;                               // kOthStages stages
    float* own_st = tile_smem + kOthStages * g.oth_floats;  // kOwnStages stages
    const int yi = threadIdx.x / (W / 2), k0 = 2 * (threadIdx.x % (W / 2));
    const int nsy = L / Y, items = nsy * (L / kTileZ);
    const uint32_t bar0 = smem_addr(bars);
    if (threadIdx.x == 0) {
        for (int q = 0; q < kOthStages + kOwnStages; ++q) mbar_init(bar0 + 8 * q);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;    // bit s: parity of stage s's next completion
    uint32_t pending = 0;  // bit s: stage s has a fill in flight (every thread tracks it)
    // other-colour plane pi of the item (plane z0 - 1 + pi, rows y0 - 1 .. y0 + Y)
    auto issue_oth = [&](int pi, int y0, int z0) {
        const int s = pi % kOthStages;
        pending |= 1u << s;
        if (threadIdx.x != 0) return;
        // the block's reads of this stage (ordered by the barrier before the
        // call) come before the bulk copy's writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bar = bar0 + 8 * s;
        mbar_expect(bar, (uint32_t)g.oth_floats * 4u);
        int zz = z0 - 1 + pi;
        zz = zz < 0 ? zz + L : (zz >= L ? zz - L : zz);
        float* dst = oth_st + s * g.oth_floats;
        for (int c = 0; c < 3; ++c) {
            const float* plane = a.oth + c * H + (long long)zz * L * W;
            float* d = dst + c * (Y + 2) * W;
            if (y0 == 0) {  // row -1 is row L-1
                bulk_load(smem_addr(d), plane + (long long)(L - 1) * W, (uint32_t)W * 4u, bar);
                bulk_load(smem_addr(d + W), plane, (uint32_t)(Y + 1) * W * 4u, bar);
            } else if (y0 + Y == L) {  // row y0 + Y is row 0
                bulk_load(smem_addr(d), plane + (long long)(y0 - 1) * W, (uint32_t)(Y + 1) * W * 4u,
                          bar);
                bulk_load(smem_addr(d + (Y + 1) * W), plane, (uint32_t)W * 4u, bar);
            } else {
                bulk_load(smem_addr(d), plane + (long long)(y0 - 1) * W, (uint32_t)(Y + 2) * W * 4u,
                          bar);
            }
        }
    };
    // own-colour plane oi of the item (plane z0 + oi, rows y0 .. y0 + Y - 1)
    auto issue_own = [&](int oi, int y0, int z0) {
        const int s = kOthStages + oi % kOwnStages;
        pending |= 1u << s;
        if (threadIdx.x != 0) return;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bar = bar0 + 8 * s;
        mbar_expect(bar, (uint32_t)g.own_floats * 4u);
        float* dst = own_st + (oi % kOwnStages) * g.own_floats;
        for (int c = 0; c < 3; ++c)
            bulk_load(smem_addr(dst + c * Y * W),
                      a.own + c * H + ((long long)(z0 + oi) * L + y0) * W, (uint32_t)Y * W * 4u, bar);
    };
    // Lane 0 of each warp polls (it observes the copy's completion for its
    // warp); the block barrier after the waits passes the outcome to every
    // thread.  A stage whose wait ran out stays marked in flight.
    auto wait_stage = [&](int s) {
        const bool ok =
            (threadIdx.x & 31) != 0 || mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
        phase ^= 1u << s;
        pending &= ~(1u << s);
        if (!ok) pending |= 1u << s;
        return ok;
    };
    float pe = 0.f, pmx = 0.f, pmy = 0.f, pmz = 0.f;
    bool failed = false;
    for (int item = blockIdx.x; item < items && !failed; item += gridDim.x) {
        const int y0 = (item % nsy) * Y, z0 = (item / nsy) * kTileZ;
        const int y = y0 + yi;
        for (int pi = 0; pi < kOthStages; ++pi) issue_oth(pi, y0, z0);
        for (int oi = 0; oi < kOwnStages; ++oi) issue_own(oi, y0, z0);
        for (int k = 0; k < kTileZ; ++k) {
            bool ok = true;
            if (k == 0) {
                ok = wait_stage(0) && ok;
                ok = wait_stage(1) && ok;
            }
            ok = wait_stage((k + 2) % kOthStages) && ok;
            ok = wait_stage(kOthStages + k % kOwnStages) && ok;
            if (__syncthreads_or(!ok)) {
                // the phase bits flipped for a completion that did not come
                phase ^= pending;
                failed = true;
                break;
            }
            const int z = z0 + k;
            const int p = (y + z + a.c) & 1;
            const float* om = oth_st + (k % kOthStages) * g.oth_floats;        // plane z - 1
            const float* oc = oth_st + ((k + 1) % kOthStages) * g.oth_floats;  // plane z
            const float* op = oth_st + ((k + 2) % kOthStages) * g.oth_floats;  // plane z + 1
            const float* ow = own_st + (k % kOwnStages) * g.own_floats;
            float hA[3], hB[3], sp[3][2], cur2[3][2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int row = c * (Y + 2) * W + (yi + 1) * W;
                const float2 cur = *reinterpret_cast<const float2*>(oc + row + k0);
                const float edge = oc[row + (p ? ((k0 + 2) & (W - 1)) : ((k0 - 1) & (W - 1)))];
                const float2 ym = *reinterpret_cast<const float2*>(oc + row - W + k0);
                const float2 yp = *reinterpret_cast<const float2*>(oc + row + W + k0);
                const float2 zm = *reinterpret_cast<const float2*>(om + row + k0);
                const float2 zp = *reinterpret_cast<const float2*>(op + row + k0);
                const float2 own = *reinterpret_cast<const float2*>(ow + c * Y * W + yi * W + k0);
                hA[c] = heis_field<3>(p ? cur.y : edge, cur.x, zm.x, zp.x, ym.x, yp.x, J);
                hB[c] = heis_field<3>(p ? edge : cur.x, cur.y, zm.y, zp.y, ym.y, yp.y, J);
                sp[c][0] = own.x;
                sp[c][1] = own.y;
                cur2[c][0] = cur.x;
                cur2[c][1] = cur.y;
            }
            const int j = (z * L + y) * W + k0;  // global colour index of column k0
            if (a.update) {
                bool changed = false;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const uint4 rnd = philox4x32_10(
                        make_uint4((uint32_t)(j + b), t, a.replica, (kSweep << 1) | (uint32_t)a.c),
                        a.rk);
                    const float* h = b ? hB : hA;
                    const float3 v = sphere_point_tab(tab, rnd.y, rnd.z);
                    changed = heis_metropolis<false>(sp[0][b], sp[1][b], sp[2][b], v, h[0], h[1],
                                                     h[2], u24(rnd.x), a.beta, renorm) ||
                              changed;
                }
                if (changed) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        *reinterpret_cast<float2*>(a.own + c * H + j) =
                            make_float2(sp[c][0], sp[c][1]);
                }
            }
            if (MEAS) {
                pe -= sp[0][0] * hA[0] + sp[1][0] * hA[1] + sp[2][0] * hA[2] + sp[0][1] * hB[0] +
                      sp[1][1] * hB[1] + sp[2][1] * hB[2];
                pmx += sp[0][0] + sp[0][1] + cur2[0][0] + cur2[0][1];
                pmy += sp[1][0] + sp[1][1] + cur2[1][0] + cur2[1][1];
                pmz += sp[2][0] + sp[2][1] + cur2[2][0] + cur2[2][1];
            }
            __syncthreads();  // the stages of plane z - 1 and of own plane z are free
            if (k + kOthStages < kTileZ + 2) issue_oth(k + kOthStages, y0, z0);
            if (k + kOwnStages < kTileZ) issue_own(k + kOwnStages, y0, z0);
        }
    }
    if (failed) {
        // a wait ran out: report it, wait (bounded again) for the copies still
        // in flight so that none lands after the block has left, then stop
        if (threadIdx.x == 0) atomicOr(&a.ctrl->error, 1u);
        for (int s = 0; s < kOthStages + kOwnStages; ++s)
            if ((pending >> s) & 1u) wait_stage(s);
        return;
    }
    if (!MEAS) return;
    Partial mine;
    mine.i0 = mine.i1 = 0;
    mine.f[0] = block_sum((double)pe, red);
    mine.f[1] = block_sum((double)pmx, red);
    mine.f[2] = block_sum((double)pmy, red);
    mine.f[3] = block_sum((double)pmz, red);
    store_partial(a.partials, mine);
}

// XY, 2D: each thread owns the column pair (2q, 2q+1), whose sites share one
// Philox block (group j >> 1).
template <bool FAST, bool HB, bool MEAS>
__global__ void __launch_bounds__(256) xy_stream(const OnArgs a)
{
    __shared__ double red[32];
    // Metropolis with accurate functions: sin and cos from the shared table
    constexpr bool TAB = !FAST && !HB;
    __shared__ float2 tab[TAB ? kTurnTab : 1];
    if (TAB) fill_turn_table(tab);
    auto sc = [&](float tt, float* sn, float* cs) {
        if (TAB) sincos_turns_tab(tab, tt, sn, cs);
        else sincos_angle<FAST>(tt, sn, cs);
    };
    auto sc_pair = [&](const float* p, long long i) {
        const float2 th = __ldg(reinterpret_cast<const float2*>(p + i));
        CS2 r;
        sc(th.x, &r.s0, &r.c0);
        sc(th.y, &r.s1, &r.c1);
        return r;
    };
    const uint32_t t = (uint32_t)a.ctrl->t;
    const int L = a.L, W = a.W, R = a.R;
    const int WP = W / 2;
    const int lane = threadIdx.x & 31;
    const long long nitems = (long long)WP * (L / R);
    const float J = a.J;
    float pe = 0.f, pmx = 0.f, pmy = 0.f;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(it % WP);
        const int m0 = (int)(it / WP) * R;
        const int k0 = 2 * q;
        const int mprev = m0 == 0 ? L - 1 : m0 - 1;
        CS2 prev = sc_pair(a.oth, (long long)mprev * W + k0);
        CS2 cur = sc_pair(a.oth, (long long)m0 * W + k0);
        float2 nxt_pf = __ldg(reinterpret_cast<const float2*>(
            a.oth + (long long)(m0 == L - 1 ? 0 : m0 + 1) * W + k0));
        float2 own_pf = *reinterpret_cast<const float2*>(a.own + (long long)m0 * W + k0);
        // angle of the x neighbour a warp-edge lane cannot get by shuffle:
        // column 2q-1 for lane 0 when p = 0, column 2q+2 for lane 31 when p = 1
        const int kl = k0 == 0 ? W - 1 : k0 - 1, kr = k0 + 2 == W ? 0 : k0 + 2;
        float edge_pf = 0.f;
        {
            const int p0 = (m0 + a.c) & 1;
            if (p0 ? lane == 31 : lane == 0)
                edge_pf = __ldg(a.oth + (long long)m0 * W + (p0 ? kr : kl));
        }
        // two rows at a time for Metropolis (their draws and sin/cos interleave);
        // the heat-bath's attempt loops do better one row at a time
#pragma unroll (HB ? 1 : 2)
        for (int r = 0; r < R; ++r) {
            const int m = m0 + r;
            const int p = (m + a.c) & 1;
            const long long j = (long long)m * W + k0;
            CS2 nxt;
            sc(nxt_pf.x, &nxt.s0, &nxt.c0);
            sc(nxt_pf.y, &nxt.s1, &nxt.c1);
            float2 th = own_pf;
            const float edge = edge_pf;
            if (r + 1 < R) {
                const int m2 = m + 2 >= L ? m + 2 - L : m + 2;
                nxt_pf = __ldg(reinterpret_cast<const float2*>(a.oth + (long long)m2 * W + k0));
                own_pf = *reinterpret_cast<const float2*>(a.own + (long long)(m + 1) * W + k0);
                const int p1 = p ^ 1;
                if (p1 ? lane == 31 : lane == 0)
                    edge_pf = __ldg(a.oth + (long long)(m + 1) * W + (p1 ? kr : kl));
            }
            // x neighbours of column 2q and 2q+1:
            //   p = 0: (2q-1, 2q) and (2q, 2q+1);  p = 1: (2q, 2q+1) and (2q+1, 2q+2)
            float ec, es;  // cos / sin of column 2q-1 (p = 0) or 2q+2 (p = 1)
            if (p == 0) {
                ec = __shfl_up_sync(0xffffffffu, cur.c1, 1);
                es = __shfl_up_sync(0xffffffffu, cur.s1, 1);
                if (lane == 0) sc(edge, &es, &ec);
            } else {
                ec = __shfl_down_sync(0xffffffffu, cur.c0, 1);
                es = __shfl_down_sync(0xffffffffu, cur.s0, 1);
                if (lane == 31) sc(edge, &es, &ec);
            }
            float hx0, hy0, hx1, hy1;
            if (p == 0) {
                hx0 = ec + cur.c0;
                hy0 = es + cur.s0;
                hx1 = cur.c0 + cur.c1;
                hy1 = cur.s0 + cur.s1;
            } else {
                hx0 = cur.c0 + cur.c1;
                hy0 = cur.s0 + cur.s1;
                hx1 = cur.c1 + ec;
                hy1 = cur.s1 + es;
            }
            hx0 = J * (hx0 + prev.c0 + nxt.c0);
            hy0 = J * (hy0 + prev.s0 + nxt.s0);
            hx1 = J * (hx1 + prev.c1 + nxt.c1);
            hy1 = J * (hy1 + prev.s1 + nxt.s1);
            float sx0, sy0, sx1, sy1;
            sc(th.x, &sy0, &sx0);
            sc(th.y, &sy1, &sx1);
            if (a.update && HB) {
                // both sites of the pair draw from the same Philox block per attempt
                const VonMises m0 = von_mises_setup(hx0, hy0, a.beta);
                const VonMises m1 = von_mises_setup(hx1, hy1, a.beta);
                bool p0 = true, p1 = true;
                uint32_t acc0 = 0u, acc1 = 0u;  // U1 outputs of the accepted attempts
                for (int at = 0; at < kVonMisesAttempts && (p0 || p1); ++at) {
                    const uint4 rnd = philox4x32_10(
                        make_uint4((uint32_t)(j >> 1), t, a.replica,
                                   ((uint32_t)at << 16) | (kSweep << 1) | (uint32_t)a.c),
                        a.rk);
                    if (p0 && von_mises_accept(m0, rnd.x, rnd.y)) {
                        acc0 = rnd.x;
                        p0 = false;
                    }
                    if (p1 && von_mises_accept(m1, rnd.z, rnd.w)) {
                        acc1 = rnd.z;
                        p1 = false;
                    }
                }
                if (!p0) th.x = von_mises_angle(m0, acc0);
                if (!p1) th.y = von_mises_angle(m1, acc1);
                sincos_angle<FAST>(th.x, &sy0, &sx0);
                sincos_angle<FAST>(th.y, &sy1, &sx1);
                *reinterpret_cast<float2*>(a.own + j) = th;
            } else if (a.update) {
                const uint4 rnd = philox4x32_10(
                    make_uint4((uint32_t)(j >> 1), t, a.replica, (kSweep << 1) | (uint32_t)a.c),
                    a.rk);
                const float n0 = u24(rnd.y), n1 = u24(rnd.w);
                float nx0, ny0, nx1, ny1;
                sc(n0, &ny0, &nx0);
                sc(n1, &ny1, &nx1);
                const float dE0 = -((nx0 - sx0) * hx0 + (ny0 - sy0) * hy0);
                const float dE1 = -((nx1 - sx1) * hx1 + (ny1 - sy1) * hy1);
                bool ch = false;
                const float w0 = boltzmann<FAST>(-a.beta * dE0);
                const float w1 = boltzmann<FAST>(-a.beta * dE1);
                if ((dE0 <= 0.f) | (u24(rnd.x) < w0)) {
                    th.x = n0;
                    sx0 = nx0;
                    sy0 = ny0;
                    ch = true;
                }
                if ((dE1 <= 0.f) | (u24(rnd.z) < w1)) {
                    th.y = n1;
                    sx1 = nx1;
                    sy1 = ny1;
                    ch = true;
                }
                if (ch) *reinterpret_cast<float2*>(a.own + j) = th;
            }
            if (MEAS) {
                pe -= sx0 * hx0 + sy0 * hy0 + sx1 * hx1 + sy1 * hy1;
                pmx += sx0 + sx1 + cur.c0 + cur.c1;
                pmy += sy0 + sy1 + cur.s0 + cur.s1;
            }
            prev = cur;
            cur = nxt;
        }
    }
    if (!MEAS) return;
    Partial mine;
    mine.i0 = mine.i1 = 0;
    mine.f[0] = block_sum((double)pe, red);
    mine.f[1] = block_sum((double)pmx, red);
    mine.f[2] = block_sum((double)pmy, red);
    mine.f[3] = 0.0;
    store_partial(a.partials, mine);
}

// Adds the partials a streaming measuring pass of nblocks blocks stored and
// closes the pass (one block of kFinishThreads; FP64 in a fixed order).
__global__ void __launch_bounds__(kFinishThreads) on_finish_kernel(const OnArgs a,
                                                                   unsigned nblocks)
{
    const Partial tot = sum_partials<true>(a.partials, nblocks);
    if (threadIdx.x == 0) on_finish(a, tot);
}

template <int NC>
__global__ void on_init_kernel(float* s0, float* s1, long long H, uint32_t replica, RoundKeys rk)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * H;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / H);
        const long long j = q % H;
        float* s = c ? s1 : s0;
        if (NC == 2) {
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)(j >> 1), 0u, replica, (kInit << 1) | (uint32_t)c), rk);
            s[j] = u24((j & 1) ? r.w : r.y);
        } else {
            const uint4 r =
                philox4x32_10(make_uint4((uint32_t)j, 0u, replica, (kInit << 1) | (uint32_t)c), rk);
            const float3 v = sphere_point<false>(r.y, r.z);
            s[j] = v.x;
            s[H + j] = v.y;
            s[2 * H + j] = v.z;
        }
    }
}

__device__ __forceinline__ int colour_of(long long i, int L)
{
    const int x = (int)(i % L);
    const long long r = i / L;
    return (x + (int)(r % L) + (int)(r / L)) & 1;
}

// natural order <-> colour arrays; `dir` 0 = scatter (nat -> colours), 1 = gather
template <int NC>
__global__ void on_layout_kernel(float* s0, float* s1, float* nat, long long N, long long H, int L,
                                 int dir)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        float* s = colour_of(i, L) ? s1 : s0;
        const long long j = i >> 1;
        if (NC == 2) {
            // natural order holds radians, the colour arrays turns
            if (dir == 0) {
                const float tr = nat[i] * (1.0f / kTwoPiF);
                s[j] = tr - floorf(tr);
            } else {
                nat[i] = kTwoPiF * s[j];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (dir == 0) s[q * H + j] = nat[3 * i + q];
                else nat[3 * i + q] = s[q * H + j];
            }
        }
    }
}

struct FBondPtrs {
    float* p[2][3];
};

__global__ void fbonds_scatter_kernel(FBondPtrs bp, const float* nat, long long N, int L, int d)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < d * N;
         k += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(k / N);
        const long long i = k % N;
        bp.p[colour_of(i, L)][mu][i >> 1] = nat[k];
    }
}

int grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > kMaxBlocks) g = kMaxBlocks;
    return (int)g;
}

OnArgs make_args(const sl_lattice* h, int c)
{
    OnArgs a;
    a.own = (float*)h->spins[c];
    a.oth = (const float*)h->spins[1 - c];
    for (int mu = 0; mu < 3; ++mu) {
        a.Jown[mu] = (const float*)h->bonds[c][mu];
        a.Joth[mu] = (const float*)h->bonds[1 - c][mu];
    }
    a.d = h->d;
    a.L = h->L;
    a.W = h->W;
    a.c = c;
    a.H = h->H;
    a.N = h->N;
    a.replica = h->replica;
    a.J = (float)h->J;
    a.ctrl = h->ctrl;
    a.partials = h->partials;
    a.measure = c == 1;
    a.update = 1;
    a.R = 1;
    a.renorm_every = h->renorm_every;
    return a;
}

// The staged 3D Heisenberg kernel: uniform J, Metropolis with the accurate
// functions, W = L/2 in {32, 64, 128, 256}.
bool tile_ok(const sl_lattice* h)
{
    const int W = h->W;
    return h->n == 3 && h->d == 3 && h->bonds[0][0] == nullptr && !h->slab &&
           (W == 32 || W == 64 || W == 128 || W == 256) && h->update == SL_UPDATE_METROPOLIS &&
           !h->fast_math;
}

cudaError_t launch_tile(const sl_lattice* h, const OnArgs& a, cudaStream_t s)
{
    const TileShape g = tile_shape(h->W);
    const size_t dyn = (size_t)(kOthStages * g.oth_floats + kOwnStages * g.own_floats) * 4;
    static bool attr_set[2] = {false, false};
    if (!attr_set[a.measure ? 1 : 0]) {
        const cudaError_t e =
            a.measure ? cudaFuncSetAttribute(heis_tile3<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 65536)
                      : cudaFuncSetAttribute(heis_tile3<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
        if (e != cudaSuccess) return e;
        attr_set[a.measure ? 1 : 0] = true;
    }
    const long long items = (long long)(h->L / g.Y) * (h->L / kTileZ);
    // resident blocks per SM (shared memory: the stages plus the 8 KiB table)
    const int fit = 3;
    const int per_sm = h->blocks_per_sm > 0 && h->blocks_per_sm < fit ? h->blocks_per_sm : fit;
    long long grid = (long long)h->sms * per_sm;
    if (grid > items) grid = items;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    if (a.measure) heis_tile3<true><<<(int)grid, kTileThreads, dyn, s>>>(a);
    else heis_tile3<false><<<(int)grid, kTileThreads, dyn, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !a.measure) return e;
    on_finish_kernel<<<1, kFinishThreads, 0, s>>>(a, (unsigned)grid);
    return cudaGetLastError();
}

bool on_stream_ok(const sl_lattice* h)
{
    if (h->bonds[0][0] != nullptr || h->kernel == 1) return false;
    if (h->n == 3) return h->W % 32 == 0;
    return h->d == 2 && h->W % 64 == 0;
}

}  // namespace

bool on_streams(const sl_lattice* h) { return on_stream_ok(h) || (h->kernel == 4 && tile_ok(h)); }

bool on_tile_ok(const sl_lattice* h) { return tile_ok(h); }

}  // namespace spinmc

extern "C" int sl_wait_selftest(void* stream, int* timed_out)
{
    using namespace spinmc;
    if (!timed_out) return fail(SL_EINVAL, "timed_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    wait_selftest_kernel<<<1, 32, 0, s>>>();
    cudaError_t e = cudaGetLastError();
    unsigned v = 2;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&v, g_wait_selftest, sizeof v, 0,
                                                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sl_wait_selftest");
    *timed_out = (int)v;
    return SL_OK;
}

namespace spinmc {

namespace {

int on_rows(const sl_lattice* h, long long cols)
{
    if (h->rows > 0) return h->rows;
    const long long cross = h->d == 3 ? h->L : 1;
    int R = 32;
    while (R > 1 && (h->L % R != 0 || cols * cross * (h->L / R) < (long long)h->sms * 1024)) R >>= 1;
    return R;
}

// kernel variant: 0 Metropolis, 1 Metropolis with intrinsics, 2 heat-bath
// (whose draws and fields use the accurate functions only)
template <int NC>
cudaError_t launch_on(const sl_lattice* h, OnArgs a, cudaStream_t s)
{
    const int var = a.update && h->update == SL_UPDATE_HEATBATH ? 2 : h->fast_math != 0;
    if (NC == 3 && h->kernel == 4 && tile_ok(h)) return launch_tile(h, a, s);
    if (on_stream_ok(h)) {
        // Heisenberg on column pairs when W % 64 == 0 (unless kernel 3 asks for
        // single columns); XY always takes pairs
        const bool pairs = NC == 2 || (h->W % 64 == 0 && h->kernel != 3);
        const long long cols = pairs ? h->W / 2 : h->W;
        a.R = on_rows(h, cols);
        const long long items = cols * (h->d == 3 ? h->L : 1) * (h->L / a.R);
        int grid = grid_for(items, 256);
        if (h->blocks_per_sm > 0 && grid > h->sms * h->blocks_per_sm)
            grid = h->sms * h->blocks_per_sm;
#define SPINMC_ON(K, ...)                                                      \
    do {                                                                       \
        if (a.measure) K<__VA_ARGS__, true><<<grid, 256, 0, s>>>(a);          \
        else K<__VA_ARGS__, false><<<grid, 256, 0, s>>>(a);                   \
    } while (0)
        if (NC == 3 && pairs) {
            if (h->d == 2) {
                if (var == 2) SPINMC_ON(heis_pair, 2, false, true);
                else if (var == 1) SPINMC_ON(heis_pair, 2, true, false);
                else SPINMC_ON(heis_pair, 2, false, false);
            } else {
                if (var == 2) SPINMC_ON(heis_pair, 3, false, true);
                else if (var == 1) SPINMC_ON(heis_pair, 3, true, false);
                else SPINMC_ON(heis_pair, 3, false, false);
            }
        } else if (NC == 3) {
            if (h->d == 2) {
                if (var == 2) SPINMC_ON(heis_stream, 2, false, true);
                else if (var == 1) SPINMC_ON(heis_stream, 2, true, false);
                else SPINMC_ON(heis_stream, 2, false, false);
            } else {
                if (var == 2) SPINMC_ON(heis_stream, 3, false, true);
                else if (var == 1) SPINMC_ON(heis_stream, 3, true, false);
                else SPINMC_ON(heis_stream, 3, false, false);
            }
        } else {
            if (var == 2) SPINMC_ON(xy_stream, false, true);
            else if (var == 1) SPINMC_ON(xy_stream, true, false);
            else SPINMC_ON(xy_stream, false, false);
        }
#undef SPINMC_ON
        if (a.measure) {
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            on_finish_kernel<<<1, kFinishThreads, 0, s>>>(a, (unsigned)grid);
        }
        return cudaGetLastError();
    }
    const long long rows = (long long)h->L * (h->d == 3 ? h->L : 1);
    const long long cap = (long long)h->sms * 8;
    int grid = (int)(rows < cap ? rows : cap);
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    if (h->d == 2) {
        if (var == 2) on_generic<NC, 2, false, true><<<grid, 128, 0, s>>>(a);
        else if (var == 1) on_generic<NC, 2, true, false><<<grid, 128, 0, s>>>(a);
        else on_generic<NC, 2, false, false><<<grid, 128, 0, s>>>(a);
    } else {
        if (var == 2) on_generic<NC, 3, false, true><<<grid, 128, 0, s>>>(a);
        else if (var == 1) on_generic<NC, 3, true, false><<<grid, 128, 0, s>>>(a);
        else on_generic<NC, 3, false, false><<<grid, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t on_init(const sl_lattice* h, cudaStream_t s)
{
    const RoundKeys rk = make_round_keys(h->init_seed);
    const int grid = grid_for(2 * h->H, 256);
    if (h->n == 2)
        on_init_kernel<2><<<grid, 256, 0, s>>>((float*)h->spins[0], (float*)h->spins[1], h->H,
                                               h->replica, rk);
    else
        on_init_kernel<3><<<grid, 256, 0, s>>>((float*)h->spins[0], (float*)h->spins[1], h->H,
                                               h->replica, rk);
    return cudaGetLastError();
}

cudaError_t on_layout(const sl_lattice* h, float* nat, int dir, cudaStream_t s)
{
    const int grid = grid_for(h->N, 256);
    if (h->n == 2)
        on_layout_kernel<2><<<grid, 256, 0, s>>>((float*)h->spins[0], (float*)h->spins[1], nat, h->N,
                                                 h->H, h->L, dir);
    else
        on_layout_kernel<3><<<grid, 256, 0, s>>>((float*)h->spins[0], (float*)h->spins[1], nat, h->N,
                                                 h->H, h->L, dir);
    return cudaGetLastError();
}

cudaError_t float_bonds_scatter(const sl_lattice* h, const float* nat, cudaStream_t s)
{
    FBondPtrs bp;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < 3; ++mu) bp.p[c][mu] = (float*)h->bonds[c][mu];
    fbonds_scatter_kernel<<<grid_for(h->d * h->N, 256), 256, 0, s>>>(bp, nat, h->N, h->L, h->d);
    return cudaGetLastError();
}

cudaError_t on_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count, cudaStream_t s)
{
    for (int64_t k = 0; k < count; ++k) {
        for (int c = 0; c < 2; ++c) {
            OnArgs a = make_args(h, c);
            a.rk = p.rk;
            a.beta = p.beta_f;
            const cudaError_t e = h->n == 2 ? launch_on<2>(h, a, s) : launch_on<3>(h, a, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t on_measure(const sl_lattice* h, cudaStream_t s)
{
    OnArgs a = make_args(h, 1);
    a.update = 0;
    a.measure = 1;
    memset(&a.rk, 0, sizeof a.rk);
    a.beta = 0.f;
    return h->n == 2 ? launch_on<2>(h, a, s) : launch_on<3>(h, a, s);  // update = 0 is safe in both
}

}  // namespace spinmc

// Particle layout on the device (structure of arrays, np entries per plane):
//   FP64: double2 xy, pxy, (eta, P_eta), q[4]    (7 planes, 112 B per particle)
//   FP32: float4 (x, y, p^x, p^y), float2 (eta, P_eta), float4 q[2]  (56 B)
//   both: int32 species, double p_T^2 at formation, int32 original index
#pragma once
#include "layout.cuh"

namespace gl {

template <typename R>
struct PState {
    R x, y, eta, px, py, Pe;
    A8<R> q;
};

template <typename R>
struct Parts;

template <>
struct Parts<double> {
    double2 *xy, *pxy, *eP, *q;
    int32_t* sp;
    double* pt0;
    int32_t* id;
    double* ptau;  // p^tau integrated from its own equation (NaN: not started)
    int64_t np;
    __device__ PState<double> load(int64_t i) const {
        PState<double> s;
        double2 a = xy[i], b = pxy[i], c = eP[i];
        s.x = a.x; s.y = a.y; s.px = b.x; s.py = b.y; s.eta = c.x; s.Pe = c.y;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            double2 v = q[(size_t)k * np + i];
            s.q.v[2 * k] = v.x;
            s.q.v[2 * k + 1] = v.y;
        }
        return s;
    }
    __device__ void store(int64_t i, const PState<double>& s) const {
        xy[i] = make_double2(s.x, s.y);
        pxy[i] = make_double2(s.px, s.py);
        eP[i] = make_double2(s.eta, s.Pe);
#pragma unroll
        for (int k = 0; k < 4; k++) q[(size_t)k * np + i] = make_double2(s.q.v[2 * k], s.q.v[2 * k + 1]);
    }
    __device__ void store_momenta(int64_t i, const PState<double>& s) const {
        pxy[i] = make_double2(s.px, s.py);
        eP[i] = make_double2(s.eta, s.Pe);
    }
    __device__ void prefetch_l2(int64_t) const {}
    // streaming (evict-first) forms for the push, which reads and writes each
    // particle once a step: the particles leave L2 to the gathered site fields
    __device__ PState<double> load_cs(int64_t i) const {
        PState<double> s;
        double2 a = __ldcs(xy + i), b = __ldcs(pxy + i), c = __ldcs(eP + i);
        s.x = a.x; s.y = a.y; s.px = b.x; s.py = b.y; s.eta = c.x; s.Pe = c.y;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            double2 v = __ldcs(q + (size_t)k * np + i);
            s.q.v[2 * k] = v.x;
            s.q.v[2 * k + 1] = v.y;
        }
        return s;
    }
    __device__ void store_cs(int64_t i, const PState<double>& s) const {
        __stcs(xy + i, make_double2(s.x, s.y));
        __stcs(pxy + i, make_double2(s.px, s.py));
        __stcs(eP + i, make_double2(s.eta, s.Pe));
#pragma unroll
        for (int k = 0; k < 4; k++) __stcs(q + (size_t)k * np + i, make_double2(s.q.v[2 * k], s.q.v[2 * k + 1]));
    }
    __device__ void store_momenta_cs(int64_t i, const PState<double>& s) const {
        __stcs(pxy + i, make_double2(s.px, s.py));
        __stcs(eP + i, make_double2(s.eta, s.Pe));
    }
};

template <>
struct Parts<float> {
    float4* xyp;
    float2* eP;
    float4* q;
    int32_t* sp;
    double* pt0;
    int32_t* id;
    float* ptau;   // p^tau integrated from its own equation (NaN: not started)
    int64_t np;
    __device__ PState<float> load(int64_t i) const {
        PState<float> s;
        float4 a = xyp[i];
        float2 c = eP[i];
        float4 q0 = q[i], q1 = q[np + i];
        s.x = a.x; s.y = a.y; s.px = a.z; s.py = a.w; s.eta = c.x; s.Pe = c.y;
        s.q.v[0] = q0.x; s.q.v[1] = q0.y; s.q.v[2] = q0.z; s.q.v[3] = q0.w;
        s.q.v[4] = q1.x; s.q.v[5] = q1.y; s.q.v[6] = q1.z; s.q.v[7] = q1.w;
        return s;
    }
    __device__ void store(int64_t i, const PState<float>& s) const {
        xyp[i] = make_float4(s.x, s.y, s.px, s.py);
        eP[i] = make_float2(s.eta, s.Pe);
        q[i] = make_float4(s.q.v[0], s.q.v[1], s.q.v[2], s.q.v[3]);
        q[np + i] = make_float4(s.q.v[4], s.q.v[5], s.q.v[6], s.q.v[7]);
    }
    __device__ void store_momenta(int64_t i, const PState<float>& s) const {
        xyp[i] = make_float4(s.x, s.y, s.px, s.py);
        eP[i] = make_float2(s.eta, s.Pe);
    }
    // streaming (evict-first) forms for the push, as for FP64
    __device__ PState<float> load_cs(int64_t i) const {
        PState<float> s;
        float4 a = __ldcs(xyp + i);
        float2 c = __ldcs(eP + i);
        float4 q0 = __ldcs(q + i), q1 = __ldcs(q + np + i);
        s.x = a.x; s.y = a.y; s.px = a.z; s.py = a.w; s.eta = c.x; s.Pe = c.y;
        s.q.v[0] = q0.x; s.q.v[1] = q0.y; s.q.v[2] = q0.z; s.q.v[3] = q0.w;
        s.q.v[4] = q1.x; s.q.v[5] = q1.y; s.q.v[6] = q1.z; s.q.v[7] = q1.w;
        return s;
    }
    __device__ void store_cs(int64_t i, const PState<float>& s) const {
        __stcs(xyp + i, make_float4(s.x, s.y, s.px, s.py));
        __stcs(eP + i, make_float2(s.eta, s.Pe));
        __stcs(q + i, make_float4(s.q.v[0], s.q.v[1], s.q.v[2], s.q.v[3]));
        __stcs(q + np + i, make_float4(s.q.v[4], s.q.v[5], s.q.v[6], s.q.v[7]));
    }
    __device__ void store_momenta_cs(int64_t i, const PState<float>& s) const {
        __stcs(xyp + i, make_float4(s.x, s.y, s.px, s.py));
        __stcs(eP + i, make_float2(s.eta, s.Pe));
    }
    // particle i's state and species requested into L2 ahead of its load
    __device__ void prefetch_l2(int64_t i) const {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(xyp + i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(eP + i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q + i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q + np + i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(sp + i));
    }
};

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R>
__host__ __device__ inline Parts<R> carve_parts(void* base, int64_t np);

template <>
__host__ __device__ inline Parts<double> carve_parts<double>(void* base, int64_t np) {
    Parts<double> p;
    char* c = (char*)base;
    p.np = np;
    p.xy = (double2*)c; c += align256(16 * np);
    p.pxy = (double2*)c; c += align256(16 * np);
    p.eP = (double2*)c; c += align256(16 * np);
    p.q = (double2*)c; c += align256(64 * np);
    p.sp = (int32_t*)c; c += align256(4 * np);
    p.pt0 = (double*)c; c += align256(8 * np);
    p.id = (int32_t*)c; c += align256(4 * np);
    p.ptau = (double*)c;
    return p;
}

template <>
__host__ __device__ inline Parts<float> carve_parts<float>(void* base, int64_t np) {
    Parts<float> p;
    char* c = (char*)base;
    p.np = np;
    p.xyp = (float4*)c; c += align256(16 * np);
    p.eP = (float2*)c; c += align256(8 * np);
    p.q = (float4*)c; c += align256(32 * np);
    p.sp = (int32_t*)c; c += align256(4 * np);
    p.pt0 = (double*)c; c += align256(8 * np);
    p.id = (int32_t*)c; c += align256(4 * np);
    p.ptau = (float*)c;
    return p;
}

}  // namespace gl

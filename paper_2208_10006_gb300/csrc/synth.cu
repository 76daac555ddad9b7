// MIMO H(f) synthesis on CUDA cores (Eq. 11-14, near-field spherical
// wavefront of Sec. I), the plain FP32 and FP64 forms.
//
// For the paths of one receiver, with first/last interaction points P1/Pm,
//   H[f,q,p] = sum_n w_n(f) exp(-j 2 pi f (dt_pn + dr_qn) / c),
//   w_n(f)   = g_n(f) exp(-j 2 pi frac(f L_n / c)),
//   dt_pn    = |T_p - P1| - |T_0 - P1|,  dr_qn = |R_q - Pm| - |R_0 - Pm|;
// a LoS path uses dlos_qp = |T_p - R_q| - |T_0 - R_0| instead of dt + dr.
// The prologue computes the element delays and w in FP64 (the large phase
// f L / c is reduced there); the summation then runs in FP32 or FP64.
#include <algorithm>

#include "sbr_internal.cuh"
#include "synth_common.cuh"

namespace sbr {

namespace {

__global__ void k_prep_delays(int32_t Pr, const int32_t* __restrict__ nb, const double* __restrict__ pts,
                              d3 T0, const double* __restrict__ R0p, const double* __restrict__ tx_elem,
                              int32_t Nt, const double* __restrict__ rx_elem, int32_t Nr,
                              double* __restrict__ dt, double* __restrict__ dr) {
    const d3 R0 = ld3(R0p);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t ne = (int64_t)Nt + Nr;
    if (t >= (int64_t)Pr * ne) return;
    int64_t n = t / ne;
    int32_t e = (int32_t)(t - n * ne);
    int m = nb[n];
    double v = 0.0;
    if (m > 0) {
        if (e < Nt) {
            d3 P1 = ld3(pts + (n * kKmax) * 3);
            v = norm(ld3(tx_elem + 3 * e) - P1) - norm(T0 - P1);
        } else {
            d3 Pm = ld3(pts + (n * kKmax + m - 1) * 3);
            v = norm(ld3(rx_elem + 3 * (e - Nt)) - Pm) - norm(R0 - Pm);
        }
    }
    if (e < Nt) dt[n * Nt + e] = v;
    else dr[n * Nr + (e - Nt)] = v;
}

__global__ void k_prep_w(int32_t Pr, int32_t F, const float2* __restrict__ g,
                         const double* __restrict__ L, const double* __restrict__ freqs,
                         double2* __restrict__ w) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Pr * F) return;
    int64_t f = t / Pr;
    int64_t n = t - f * Pr;
    double cyc = freqs[f] * L[n] / kC0;
    double fr = cyc - floor(cyc);
    double s, c;
    sincospi(-2.0 * fr, &s, &c);
    float2 gg = g[n * F + f];
    w[f * Pr + n] = make_double2(gg.x * c - gg.y * s, gg.x * s + gg.y * c);
}

__global__ void k_prep_los(d3 T0, const double* __restrict__ R0p, const double* __restrict__ tx_elem,
                           int32_t Nt, const double* __restrict__ rx_elem, int32_t Nr,
                           double* __restrict__ dlos) {
    const d3 R0 = ld3(R0p);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Nr * Nt) return;
    int64_t q = t / Nt, p = t - q * Nt;
    dlos[t] = norm(ld3(tx_elem + 3 * p) - ld3(rx_elem + 3 * q)) - norm(T0 - R0);
}

template <class R>
struct Cplx;
template <>
struct Cplx<float> { using T = float2; };
template <>
struct Cplx<double> { using T = double2; };

__device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }

template <class R>
__global__ void k_convert(const double* __restrict__ in, R* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (R)in[i];
}

template <class R>
__global__ void k_convert2(const double2* __restrict__ in, typename Cplx<R>::T* __restrict__ out,
                           int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { out[i].x = (R)in[i].x; out[i].y = (R)in[i].y; }
}

constexpr int kSynthThreads = 128;

template <class R>
__global__ void __launch_bounds__(kSynthThreads)
k_synth(int32_t F, int32_t Nr, int32_t Nt, int32_t Pr, const int32_t* __restrict__ nb0,
        const double* __restrict__ freqs,
        const typename Cplx<R>::T* __restrict__ w, const R* __restrict__ dt, const R* __restrict__ dr,
        const R* __restrict__ dlos, float2* __restrict__ H) {
    using C2 = typename Cplx<R>::T;
    __shared__ C2 s_w[kSynthThreads];
    __shared__ R s_dr[kSynthThreads];
    const int32_t p = blockIdx.x * kSynthThreads + threadIdx.x;
    const int32_t q = blockIdx.y;
    const int32_t f = blockIdx.z;
    const R foc = (R)(freqs[f] / kC0);
    const int32_t los = (Pr > 0 && *nb0 == 0) ? 0 : -1;
    const bool act = p < Nt;
    R acc_re = 0, acc_im = 0;
    for (int32_t n0 = 0; n0 < Pr; n0 += kSynthThreads) {
        int32_t n = n0 + threadIdx.x;
        if (n < Pr) {
            s_w[threadIdx.x] = w[(int64_t)f * Pr + n];
            s_dr[threadIdx.x] = dr[(int64_t)n * Nr + q];
        }
        __syncthreads();
        int32_t cnt = min(kSynthThreads, Pr - n0);
        if (act) {
            for (int32_t k = 0; k < cnt; ++k) {
                int32_t nn = n0 + k;
                R delay = nn == los ? dlos[(int64_t)q * Nt + p] : dt[(int64_t)nn * Nt + p] + s_dr[k];
                R s, c;
                sincospi_((R)-2 * foc * delay, &s, &c);
                C2 ww = s_w[k];
                acc_re += ww.x * c - ww.y * s;
                acc_im += ww.x * s + ww.y * c;
            }
        }
        __syncthreads();
    }
    if (act) H[((int64_t)f * Nr + q) * Nt + p] = make_float2((float)acc_re, (float)acc_im);
}

inline unsigned nb256(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

// per-element reception: element delays of every path (FP64),
//   dt_np = |T_p - R_q| - L_n for the LoS path of element q (so that L_n + dt_np
//   is the exact element-pair distance), |T_p - P1| - |T_0 - P1| otherwise
__global__ void k_el_delays(int64_t P, const int32_t* __restrict__ rx, const int32_t* __restrict__ nb,
                            const double* __restrict__ pts, const double* __restrict__ L, d3 T0,
                            const double* __restrict__ rx_xyz, const double* __restrict__ tx_elem, int32_t Nt,
                            double* __restrict__ dt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * Nt) return;
    int64_t n = t / Nt;
    int32_t p = (int32_t)(t - n * Nt);
    d3 Tp = ld3(tx_elem + 3 * p);
    double v;
    if (nb[n] == 0) {
        v = norm(Tp - ld3(rx_xyz + 3 * rx[n])) - L[n];
    } else {
        d3 P1 = ld3(pts + (n * kKmax) * 3);
        v = norm(Tp - P1) - norm(T0 - P1);
    }
    dt[t] = v;
}

// H[f, q, :] = sum over element q's own paths n of w_n(f) exp(-j 2 pi f dt_np / c)
template <class R>
__global__ void __launch_bounds__(kSynthThreads)
k_synth_el(int32_t F, int32_t Nq, int32_t Nt, int64_t P, const int32_t* __restrict__ rx_off,
           const double* __restrict__ freqs, const typename Cplx<R>::T* __restrict__ w,
           const R* __restrict__ dt, float2* __restrict__ H) {
    using C2 = typename Cplx<R>::T;
    __shared__ C2 s_w[kSynthThreads];
    const int32_t p = blockIdx.x * kSynthThreads + threadIdx.x;
    const int32_t q = blockIdx.y;
    const int32_t f = blockIdx.z;
    const R foc = (R)(freqs[f] / kC0);
    const bool act = p < Nt;
    const int32_t a0 = rx_off[q], a1 = rx_off[q + 1];
    R acc_re = 0, acc_im = 0;
    for (int32_t n0 = a0; n0 < a1; n0 += kSynthThreads) {
        int32_t n = n0 + threadIdx.x;
        if (n < a1) s_w[threadIdx.x] = w[(int64_t)f * P + n];
        __syncthreads();
        int32_t cnt = min(kSynthThreads, a1 - n0);
        if (act) {
            for (int32_t k = 0; k < cnt; ++k) {
                R s, c;
                sincospi_((R)-2 * foc * dt[(int64_t)(n0 + k) * Nt + p], &s, &c);
                C2 ww = s_w[k];
                acc_re += ww.x * c - ww.y * s;
                acc_im += ww.x * s + ww.y * c;
            }
        }
        __syncthreads();
    }
    if (act) H[((int64_t)f * Nq + q) * Nt + p] = make_float2((float)acc_re, (float)acc_im);
}

}  // namespace

sbr_status synth_elements_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                              const double* tx_elem, int32_t Nt, bool fp64, float2* H, cudaStream_t s) {
    const int64_t P = pl->P;
    const int32_t Nq = pl->n_rx;
    const int64_t Pp = std::max<int64_t>(P, 1);
    double* dt;
    double2* w;
    SBR_TRY(dalloc_n(&dt, (size_t)Pp * Nt, s));
    SBR_TRY(dalloc_n(&w, (size_t)Pp * F, s));
    if (P > 0) {
        d3 T0 = mk3(pl->tx[0], pl->tx[1], pl->tx[2]);
        ::sbr::note_launch(), k_el_delays<<<nb256(P * Nt), 256, 0, s>>>(P, pl->rx, pl->nb, pl->pts, pl->L, T0,
                                                                       pl->rx_xyz, tx_elem, Nt, dt);
        ::sbr::note_launch(), k_prep_w<<<nb256(P * F), 256, 0, s>>>((int32_t)P, F, g, pl->L, freqs, w);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    dim3 grid((unsigned)((Nt + kSynthThreads - 1) / kSynthThreads), (unsigned)Nq, (unsigned)F);
    if (fp64) {
        ::sbr::note_launch(), k_synth_el<double><<<grid, kSynthThreads, 0, s>>>(F, Nq, Nt, Pp, pl->rx_off, freqs, w,
                                                                               dt, H);
    } else {
        float* dtf;
        float2* wf;
        SBR_TRY(dalloc_n(&dtf, (size_t)Pp * Nt, s));
        SBR_TRY(dalloc_n(&wf, (size_t)Pp * F, s));
        ::sbr::note_launch(), k_convert<float><<<nb256(Pp * Nt), 256, 0, s>>>(dt, dtf, Pp * Nt);
        ::sbr::note_launch(), k_convert2<float><<<nb256(Pp * F), 256, 0, s>>>(w, wf, Pp * F);
        ::sbr::note_launch(), k_synth_el<float><<<grid, kSynthThreads, 0, s>>>(F, Nq, Nt, Pp, pl->rx_off, freqs, wf,
                                                                              dtf, H);
        dfree(dtf, s);
        dfree(wf, s);
    }
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(dt, s);
    dfree(w, s);
    return SBR_OK;
}

sbr_status synth_prepare(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                         const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                         int32_t rx_index, SynthPrep* sp, cudaStream_t s) {
    const int32_t o0 = pl->h_rx_off[rx_index], o1 = pl->h_rx_off[rx_index + 1];
    sp->Pr = o1 - o0;
    sp->off = o0;
    // the LoS path (no reflection) sorts first among a receiver's paths; the
    // kernels read its reflection count and the receiver reference on the device
    sp->nb0 = pl->nb + o0;
    const int32_t Pr = std::max(sp->Pr, 1);
    d3 T0 = mk3(pl->tx[0], pl->tx[1], pl->tx[2]);
    const double* R0 = pl->rx_xyz + 3 * rx_index;
    SBR_TRY(dalloc_n(&sp->dt, (size_t)Pr * Nt, s));
    SBR_TRY(dalloc_n(&sp->dr, (size_t)Pr * Nr, s));
    SBR_TRY(dalloc_n(&sp->w, (size_t)Pr * F, s));
    SBR_TRY(dalloc_n(&sp->dlos, (size_t)Nr * Nt, s));
    if (sp->Pr > 0) {
        int64_t ne = (int64_t)sp->Pr * (Nt + Nr);
        ::sbr::note_launch(), k_prep_delays<<<nb256(ne), 256, 0, s>>>(sp->Pr, pl->nb + o0, pl->pts + (int64_t)o0 * kKmax * 3,
                                                T0, R0, tx_elem, Nt, rx_elem, Nr, sp->dt, sp->dr);
        ::sbr::note_launch(), k_prep_w<<<nb256((int64_t)sp->Pr * F), 256, 0, s>>>(sp->Pr, F, g + (int64_t)o0 * F,
                                                            pl->L + o0, freqs, sp->w);
    }
    ::sbr::note_launch(), k_prep_los<<<nb256((int64_t)Nr * Nt), 256, 0, s>>>(T0, R0, tx_elem, Nt, rx_elem, Nr, sp->dlos);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

void synth_release(SynthPrep* sp, cudaStream_t s) {
    if (sp->dt) dfree(sp->dt, s);
    if (sp->dr) dfree(sp->dr, s);
    if (sp->w) dfree(sp->w, s);
    if (sp->dlos) dfree(sp->dlos, s);
    *sp = SynthPrep{};
}

sbr_status synth_simt_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                          const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                          int32_t rx_index, bool fp64, float2* H, cudaStream_t s) {
    SynthPrep sp;
    SBR_TRY(synth_prepare(pl, g, freqs, F, tx_elem, Nt, rx_elem, Nr, rx_index, &sp, s));
    dim3 grid((unsigned)((Nt + kSynthThreads - 1) / kSynthThreads), (unsigned)Nr, (unsigned)F);
    const int32_t Pr = std::max(sp.Pr, 1);
    if (fp64) {
        ::sbr::note_launch(), k_synth<double><<<grid, kSynthThreads, 0, s>>>(F, Nr, Nt, sp.Pr, sp.nb0, freqs, sp.w, sp.dt,
                                                       sp.dr, sp.dlos, H);
        SBR_TRY_CUDA(cudaGetLastError());
    } else {
        float *dt, *dr, *dl;
        float2* w;
        SBR_TRY(dalloc_n(&dt, (size_t)Pr * Nt, s));
        SBR_TRY(dalloc_n(&dr, (size_t)Pr * Nr, s));
        SBR_TRY(dalloc_n(&dl, (size_t)Nr * Nt, s));
        SBR_TRY(dalloc_n(&w, (size_t)Pr * F, s));
        ::sbr::note_launch(), k_convert<float><<<nb256((int64_t)Pr * Nt), 256, 0, s>>>(sp.dt, dt, (int64_t)Pr * Nt);
        ::sbr::note_launch(), k_convert<float><<<nb256((int64_t)Pr * Nr), 256, 0, s>>>(sp.dr, dr, (int64_t)Pr * Nr);
        ::sbr::note_launch(), k_convert<float><<<nb256((int64_t)Nr * Nt), 256, 0, s>>>(sp.dlos, dl, (int64_t)Nr * Nt);
        ::sbr::note_launch(), k_convert2<float><<<nb256((int64_t)Pr * F), 256, 0, s>>>(sp.w, w, (int64_t)Pr * F);
        ::sbr::note_launch(), k_synth<float><<<grid, kSynthThreads, 0, s>>>(F, Nr, Nt, sp.Pr, sp.nb0, freqs, w, dt, dr, dl, H);
        SBR_TRY_CUDA(cudaGetLastError());
        dfree(dt, s); dfree(dr, s); dfree(dl, s); dfree(w, s);
    }
    synth_release(&sp, s);
    return SBR_OK;
}

}  // namespace sbr

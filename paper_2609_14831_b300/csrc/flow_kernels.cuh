// flow_kernels.cuh -- device-side Dormand-Prince step control.
//
// The adaptive integrator runs without host round trips: the step size, the
// flow coordinate, the accept/reject decision and the status live in a
// device-resident control block that one thread updates after each attempt;
// every other kernel of an attempt reads it.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace cut {
namespace k {

struct Control {
    double s, ds, s1, rtol, atol;
    unsigned long long err_bits;  // max error ratio of the attempt (as ordered bits)
    int nonfinite;
    int done, status, accepted;
    long long steps, rejects, attempts, max_steps, n_replay;
    long long pause_after;   // > 0: stop (status OK, not finished) after this many attempts
    int paused;
};

// r = max_k |ds sum_i e_i K_i[k]| / (atol + rtol max(|y_k|, |y5_k|))
struct ErrTerms {
    const double *K[7];
    double e[7];
};

__global__ void dp_error(ErrTerms et, const double *__restrict__ y, const double *__restrict__ y5,
                         int64_t len, Control *ctl) {
    pdl_enter();
    __shared__ double red[32];
    if (ctl->done) return;
    const double ds = ctl->ds, rtol = ctl->rtol, atol = ctl->atol;
    double m = 0.0;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        double err = 0.0;
#pragma unroll
        for (int s = 0; s < 7; s++)
            if (et.e[s] != 0.0) err += (ds * et.e[s]) * et.K[s][i];
        double sc = atol + rtol * fmax(fabs(y[i]), fabs(y5[i]));
        double r = fabs(err) / sc;
        if (!(r == r) || !isfinite(y5[i])) bad = 1;
        else m = fmax(m, r);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) atomicMax(&ctl->err_bits, (unsigned long long)__double_as_longlong(v));
    }
    if (bad && (threadIdx.x & 31) == 0) atomicExch(&ctl->nonfinite, 1);
}

// One thread: accept/reject, next step size, termination.
__global__ void dp_control(Control *ctl, const double *replay, double *record, long long record_cap) {
    pdl_enter();
    if (ctl->done) { ctl->accepted = 0; return; }
    const double r = __longlong_as_double((long long)ctl->err_bits);
    const bool replaying = replay != nullptr;
    double fac;
    int acc;
    if (ctl->nonfinite) {
        ctl->status = 7;  // CUT_ERR_NONFINITE
        ctl->done = 1;
        ctl->accepted = 0;
        return;
    }
    if (replaying) {
        acc = 1;
        fac = 1.0;
    } else {
        acc = r <= 1.0;
        if (acc) fac = r == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(r, -0.2)));
        else fac = fmin(1.0, fmax(0.2, 0.9 * pow(r, -0.2)));
    }
    ctl->accepted = acc;
    ctl->attempts++;
    if (acc) {
        ctl->s += ctl->ds;
        if (record && ctl->steps < record_cap) record[ctl->steps] = ctl->ds;
        ctl->steps++;
    } else {
        ctl->rejects++;
    }
    ctl->err_bits = 0ull;
    if (replaying) {
        if (ctl->steps >= ctl->n_replay) ctl->done = 1;
        else ctl->ds = replay[ctl->steps];
        return;
    }
    double ds = ctl->ds * fac;
    if (!(ctl->s < ctl->s1)) { ctl->done = 1; return; }
    ds = fmin(ds, ctl->s1 - ctl->s);
    if (ds < 1e-14 * fmax(1.0, fabs(ctl->s))) { ctl->status = 8; ctl->done = 1; return; }  // STEP_UNDERFLOW
    ctl->ds = ds;
    if (ctl->attempts >= ctl->max_steps) { ctl->status = 9; ctl->done = 1; return; }      // MAX_STEPS
    if (ctl->pause_after > 0 && ctl->attempts >= ctl->pause_after) { ctl->paused = 1; ctl->done = 1; }
}

// After control: if the attempt was accepted, y <- y5 and K1 <- K7 (FSAL).
__global__ void dp_accept(const Control *ctl, double *__restrict__ y, const double *__restrict__ y5,
                          double *__restrict__ k1, const double *__restrict__ k7, int64_t len) {
    pdl_enter();
    if (!ctl->accepted) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        y[i] = y5[i];
        k1[i] = k7[i];
    }
}

// Non-finite scan of a state (RK4 end check).
__global__ void scan_nonfinite(const double *__restrict__ y, int64_t len, int *flag) {
    pdl_enter();
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(y[i])) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

}  // namespace k
}  // namespace cut

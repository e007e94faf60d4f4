// Error control of the outer iteration (Sec. 2.6, Eq. 20-21) on the device.
//
// delta_cell = max_c |e_new - e_old| / max(e_old, e_med), e_med the lower
// median of e_old over all cells; delta_tot = 2 |sum e_new - sum e_old| /
// (sum e_new + sum e_old) (uniform cells, so dV cancels).  The median is
// found by an 8-pass radix select over the bit patterns of the
// (non-negative) FP64 values, 8 bits per pass, with no host round trip
// between passes.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tr_internal.cuh"

namespace tr {
namespace {

struct SelectState {
    unsigned long long prefix;              // digits fixed so far
    unsigned long long rank;                // rank still to find inside the current bucket
    unsigned long long dmax;                // delta_cell as the bits of a non-negative double
    double sum_new, sum_old;
    unsigned int hist[256];
};

__global__ void k_sel_init(SelectState* s, unsigned long long rank) {
    if (threadIdx.x == 0) {
        s->prefix = 0ull; s->rank = rank; s->dmax = 0ull; s->sum_new = 0.0; s->sum_old = 0.0;
    }
    for (int d = threadIdx.x; d < 256; d += blockDim.x) s->hist[d] = 0u;
}

// histogram of digit `shift` among values whose higher digits equal the prefix
__global__ void k_sel_hist(const double* v, int64_t n, SelectState* s, int shift) {
    __shared__ unsigned int h[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0u;
    __syncthreads();
    const unsigned long long hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    const unsigned long long prefix = s->prefix;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(v[i]);
        if ((key & hi_mask) == (prefix & hi_mask)) atomicAdd(&h[(key >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
        if (h[d]) atomicAdd(&s->hist[d], h[d]);
}

// pick the digit holding the wanted rank, then clear the histogram
__global__ void k_sel_pick(SelectState* s, int shift) {
    if (threadIdx.x == 0) {
        unsigned long long r = s->rank;
        int d = 0;
        for (; d < 255; ++d) {
            if (r < s->hist[d]) break;
            r -= s->hist[d];
        }
        s->rank = r;
        s->prefix |= (unsigned long long)d << shift;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) s->hist[d] = 0u;
}

__global__ void k_delta(const double* e_new, const double* e_old, int64_t n, SelectState* s) {
    __shared__ unsigned long long wmax[32];
    __shared__ double wn[32], wo[32];
    const double med = __longlong_as_double((long long)s->prefix);
    unsigned long long m = 0ull;
    double sn = 0.0, so = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = e_new[i], b = e_old[i];
        const double norm = fmax(b, med);
        const double diff = fabs(a - b);
        const double term = (norm > 0.0) ? diff / norm : (diff > 0.0 ? INFINITY : 0.0);
        m = max(m, (unsigned long long)__double_as_longlong(term));
        sn += a;
        so += b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        so += __shfl_xor_sync(0xffffffffu, so, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { wmax[w] = m; wn[w] = sn; wo[w] = so; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { m = max(m, wmax[k]); sn += wn[k]; so += wo[k]; }
        m = max(m, wmax[0]);
        atomicMax(&s->dmax, m);
        atomicAdd(&s->sum_new, sn);
        atomicAdd(&s->sum_old, so);
    }
}

}  // namespace

size_t delta_scratch_bytes() { return sizeof(SelectState); }

tr_status delta_compute(const double* e_new, const double* e_old, int64_t n, int mode, void* scratch, double* out,
                        cudaStream_t st) {
    SelectState* s = static_cast<SelectState*>(scratch);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    k_sel_init<<<1, 256, 0, st>>>(s, (unsigned long long)((n - 1) / 2));
    if (mode == 0)
        for (int shift = 56; shift >= 0; shift -= 8) {
            k_sel_hist<<<blocks, 256, 0, st>>>(e_old, n, s, shift);
            k_sel_pick<<<1, 256, 0, st>>>(s, shift);
        }
    k_delta<<<blocks, 256, 0, st>>>(e_new, e_old, n, s);
    tr_status rc = cuda_check(cudaGetLastError(), "delta kernels");
    if (rc != TR_OK) return rc;
    unsigned long long dmax = 0ull;
    double sums[2] = {0.0, 0.0};
    rc = cuda_check(cudaMemcpyAsync(&dmax, &s->dmax, sizeof dmax, cudaMemcpyDeviceToHost, st), "delta copy");
    if (rc == TR_OK) rc = cuda_check(cudaMemcpyAsync(sums, &s->sum_new, sizeof sums, cudaMemcpyDeviceToHost, st), "sums copy");
    if (rc == TR_OK) rc = cuda_check(cudaStreamSynchronize(st), "delta kernels");
    if (rc != TR_OK) return rc;
    if (mode == 0) {
        double d;
        memcpy(&d, &dmax, sizeof d);
        *out = d;
    } else {
        const double tot = sums[0] + sums[1];
        *out = tot == 0.0 ? 0.0 : std::fabs(2.0 * (sums[0] - sums[1]) / tot);
    }
    return TR_OK;
}

}  // namespace tr

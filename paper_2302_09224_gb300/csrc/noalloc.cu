// noalloc.cu -- hisq_dslash_noalloc: the stencil entry point for callers that
// must not allocate device memory.  Its scratch (the input, xpay and output
// fields in the storage format and a non-finite counter) is one file-scope
// device array sized for at most HISQ_NOALLOC_MAX_SITES sites per parity;
// every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace hisq {

namespace {

constexpr int64_t kMaxSites = HISQ_NOALLOC_MAX_SITES;
constexpr size_t kFieldBytes = (size_t)48 * 2 * kMaxSites;  // one full-lattice field, widest format
constexpr size_t kScratchBytes = 3 * kFieldBytes + 256;

static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex addr_mu;
char *addr_of[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device (host code only holds a stand-in for the symbol).
hisq_status scratch_address(hisq_ctx *c, char **out)
{
    if (c->device < 0 || c->device >= kMaxDevices) return fail(c, HISQ_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(addr_mu);
    if (!addr_of[c->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(c, e, "cudaGetSymbolAddress(noalloc scratch)");
        addr_of[c->device] = static_cast<char *>(p);
    }
    *out = addr_of[c->device];
    return HISQ_OK;
}

}  // namespace

}  // namespace hisq

using namespace hisq;

extern "C" hisq_status hisq_dslash_noalloc(hisq_ctx *c, const hisq_gauge *g, hisq_prec prec, int out_parity,
                                           double a, const double *xpay_in, const double *in, double *out,
                                           void *stream)
{
    if (!c || !g || !in || !out) return fail(c, HISQ_EINVAL, "hisq_dslash_noalloc: null argument");
    if (out_parity < 0 || out_parity > 2) return fail(c, HISQ_EINVAL, "out_parity must be 0, 1 or 2");
    const bool xpay = a != 0.0;
    if (xpay && !xpay_in) return fail(c, HISQ_EINVAL, "xpay_in is required when a != 0");
    const int64_t vh = g->geom.vh;
    if (vh > kMaxSites)
        return fail(c, HISQ_EINVAL, "hisq_dslash_noalloc: %lld sites per parity exceed its fixed scratch (%lld)",
                    (long long)vh, (long long)kMaxSites);
    if (c->device < 0 || c->device >= kMaxDevices) return fail(c, HISQ_EINVAL, "device index out of range");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash_noalloc: cudaSetDevice");
    cudaStream_t s = pick_stream(c, stream);
    // the counter read-back and the synchronisation below cannot be captured
    if (stream_capturing(s))
        return fail(c, HISQ_EINVAL, "hisq_dslash_noalloc cannot be called while its stream is being captured");
    GaugeView gv{};
    hisq_status st = gauge_view_existing(c, g, prec, &gv);
    if (st) return st;
    char *sc = nullptr;
    st = scratch_address(c, &sc);
    if (st) return st;
    const int nhalf = out_parity == 2 ? 2 : 1;
    const size_t bs = spinor_field_bytes(prec.spinor, vh);
    char *in_s = sc, *y_s = sc + kFieldBytes, *out_s = sc + 2 * kFieldBytes;
    int *bad = reinterpret_cast<int *>(sc + 3 * kFieldBytes);
    // the array keeps the previous call's contents: the counter starts at zero
    e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash_noalloc");
    for (int h = 0; h < nhalf; h++) {
        launch_pack_spinor(prec.spinor, vh, in + h * vh * 6, in_s + h * bs, bad, s);
        c->launches++;
        if (xpay) {
            launch_pack_spinor(prec.spinor, vh, xpay_in + h * vh * 6, y_s + h * bs, bad, s);
            c->launches++;
        }
    }
    int bad_in = 0;
    e = cudaMemcpyAsync(&bad_in, bad, sizeof bad_in, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash_noalloc pack");
    if (bad_in) return fail(c, HISQ_EINVAL, "non-finite input spinor");
    for (int h = 0; h < nhalf; h++) {
        const int po = out_parity == 2 ? h : out_parity;
        const int oi = out_parity == 2 ? po : 0, ii = out_parity == 2 ? 1 - po : 0;
        DslashArgs da{};
        da.g = g->geom;
        da.gv = gv;
        da.out_parity = po;
        da.in = in_s + ii * bs;
        da.out = out_s + oi * bs;
        da.y = xpay ? y_s + oi * bs : nullptr;
        da.a = a;
        da.sign = xpay ? -1 : 1;
        da.xpay = xpay ? 1 : 0;
        da.err = bad;
        da.fin = FIN_NONE;
        if (!launch_dslash(prec.gauge, prec.spinor, prec.compute, prec.long_recon, false, da, s))
            return fail(c, HISQ_EINVAL, "no stencil kernel for this triplet");
        c->launches++;
    }
    for (int h = 0; h < nhalf; h++) {
        launch_unpack_spinor(prec.spinor, prec.compute, vh, out_s + h * bs, out + h * vh * 6, s);
        c->launches++;
    }
    // the stencil flags output sites it could not store
    int bad_out = 0;
    e = cudaMemcpyAsync(&bad_out, bad, sizeof bad_out, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash_noalloc");
    if (bad_out)
        return fail(c, HISQ_ERANGE,
                    "hisq_dslash_noalloc: output sites not storable in the spinor format (overflow or beyond its "
                    "exponent range)");
    return HISQ_OK;
}

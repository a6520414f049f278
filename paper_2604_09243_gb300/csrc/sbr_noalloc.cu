// sbr_noalloc.cu -- allocation-free variant of the PO ray-tube sum.
//
// sbr_po_integrate keeps its scratch (tube blocks, frequency table, FP64
// partial sums) in buffers the context allocates. Some callers cannot allocate
// device memory at the point where they need the sum: plug-ins that run inside
// a host application which owns and budgets all device memory (the host hands
// them buffers and forbids their own allocations), or latency-critical loops
// that must not call into the allocator, whose calls can synchronise the
// device. This entry point runs the same reduction kernels with all scratch in
// one file-scope device array of fixed size, so it never allocates: the caller
// passes the records and the output buffers.
//
// The array lives in every device that loads the library until the process
// exits. Its device address is looked up once per device, the first time the
// entry point runs with that device current (make that first call before any
// stream capture). All calls share the array: calls that overlap on the GPU
// (different streams, different host threads) race on it, so order them. The
// small tables are staged in host arrays under one lock and copied from
// pageable memory, so a call can wait for work already queued on its stream,
// and calls from several host threads take turns.
#include <math.h>
#include <string.h>

#include <mutex>

#include "sbr.h"
#include "sbr_internal.h"

namespace sbr {
void set_static_error(const char* msg);  // message read back by sbr_last_error(NULL)
}

using namespace sbr;

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kItem = 1024;  // tubes per block, as in sbr_po_integrate
constexpr int kMaxDevices = 64;

// layout of the static scratch (bytes)
constexpr size_t kItemsBytes = sizeof(PoItem) * SBR_NOALLOC_MAX_ITEMS;
constexpr size_t kOffBytes = sizeof(PoAngle) * SBR_NOALLOC_MAX_ANGLES;
constexpr size_t kFreqBytes = sizeof(float4) * SBR_NOALLOC_MAX_FREQ;
constexpr size_t kKfBytes = sizeof(double) * SBR_NOALLOC_MAX_FREQ;
constexpr size_t kPartialBytes = SBR_NOALLOC_PARTIAL_BYTES;
constexpr size_t kOffItems = 0;
constexpr size_t kOffOff = kOffItems + ((kItemsBytes + 255) & ~size_t(255));
constexpr size_t kOffFreq = kOffOff + ((kOffBytes + 255) & ~size_t(255));
constexpr size_t kOffKf = kOffFreq + ((kFreqBytes + 255) & ~size_t(255));
constexpr size_t kOffPartial = kOffKf + ((kKfBytes + 255) & ~size_t(255));
constexpr size_t kScratchBytes = kOffPartial + kPartialBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// host side: per-device address of g_scratch and one staging area for the
// small tables (copied into g_scratch before each launch)
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
PoItem g_items[SBR_NOALLOC_MAX_ITEMS];
PoAngle g_angles[SBR_NOALLOC_MAX_ANGLES];
float4 g_freq[SBR_NOALLOC_MAX_FREQ];
double g_kf[SBR_NOALLOC_MAX_FREQ];

int reject(int code, const char* msg)
{
    set_static_error(msg);
    return code;
}

}  // namespace

extern "C" int sbr_po_integrate_noalloc(const void* records, const int64_t* rec_offsets, int64_t n_angles,
                                        const double* freq_hz, int64_t n_freq, int pol_mask, int po_mode,
                                        double* E_re_im, double* rcs_dbsm, void* cuda_stream)
{
    if (!records || !rec_offsets || !freq_hz || (!E_re_im && !rcs_dbsm))
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: null pointer");
    if (n_angles < 1 || n_angles > SBR_NOALLOC_MAX_ANGLES)
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: n_angles must be 1..SBR_NOALLOC_MAX_ANGLES (4096)");
    if (n_freq < 1 || n_freq > SBR_NOALLOC_MAX_FREQ)
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: n_freq must be 1..SBR_NOALLOC_MAX_FREQ (256)");
    if (pol_mask <= 0 || pol_mask > 15)
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: pol_mask must select HH/VV/HV/VH");
    const int form = po_mode & 15, prec = po_mode & ~15;
    if ((form != SBR_PO_VECTOR && form != SBR_PO_PAPER_SCALAR) ||
        (prec != SBR_PHASE_COMPENSATED && prec != SBR_PHASE_FP32 && prec != SBR_PHASE_FP64))
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: unknown po_mode");
    for (int64_t f = 0; f < n_freq; ++f)
        if (!(freq_hz[f] > 0.0)) return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: frequencies must be > 0");
    if (rec_offsets[0] != 0) return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: rec_offsets[0] must be 0");
    for (int64_t a = 0; a < n_angles; ++a)
        if (rec_offsets[a + 1] < rec_offsets[a])
            return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: rec_offsets must not decrease");

    PoArgs pa;
    memset(&pa, 0, sizeof(pa));
    for (int q = 0; q < 4; ++q)
        if (pol_mask & (1 << q)) pa.pol_sel[pa.n_pol++] = q;
    pa.scalar = form == SBR_PO_PAPER_SCALAR;
    pa.phase_mode = prec == SBR_PHASE_COMPENSATED ? 0 : (prec == SBR_PHASE_FP32 ? 1 : 2);

    std::lock_guard<std::mutex> lock(g_mu);
    // blocks of at most kItem tubes per aspect
    long long n_items = 0;
    for (int64_t a = 0; a < n_angles; ++a) {
        const long long cnt = rec_offsets[a + 1] - rec_offsets[a];
        n_items += (cnt + kItem - 1) / kItem;
    }
    if (n_items > SBR_NOALLOC_MAX_ITEMS)
        return reject(SBR_ERR_ARG, "sbr_po_integrate_noalloc: more than SBR_NOALLOC_MAX_ITEMS blocks of 1024 tubes");
    if ((size_t)n_items * (size_t)n_freq * (size_t)pa.n_pol * 2 * sizeof(double) > kPartialBytes)
        return reject(SBR_ERR_ARG,
                      "sbr_po_integrate_noalloc: blocks x n_freq x n_pol x 16 B exceeds SBR_NOALLOC_PARTIAL_BYTES");
    int ni = 0;
    for (int64_t a = 0; a < n_angles; ++a) {
        PoAngle& A = g_angles[a];
        A.item_begin = ni;
        A.f0 = 0;
        A.nf = (int)n_freq;
        A.out_row = a * n_freq;
        A.part = 0;
        for (long long r = rec_offsets[a]; r < rec_offsets[a + 1]; r += kItem) {
            g_items[ni].angle = (int)a;
            g_items[ni].first = r;
            g_items[ni].count = (int)(rec_offsets[a + 1] - r < kItem ? rec_offsets[a + 1] - r : kItem);
            g_items[ni].f0 = 0;
            g_items[ni].nf = (int)n_freq;
            g_items[ni].part = (long long)ni * n_freq * 2 * pa.n_pol;
            ++ni;
        }
        A.item_end = ni;
    }
    for (int64_t f = 0; f < n_freq; ++f) {
        const double kappa = freq_hz[f] / kC0;
        const float kh = (float)kappa;
        g_freq[f] = make_float4(kh, (float)(kappa - (double)kh), (float)(2.0 * kPi * freq_hz[f] / kC0), 0.f);
        g_kf[f] = 2.0 * kPi * freq_hz[f] / kC0;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(SBR_ERR_CUDA, "sbr_po_integrate_noalloc: no current CUDA device");
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return reject(SBR_ERR_CUDA, "sbr_po_integrate_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        g_addr[dev] = p;
    }
    char* base = (char*)g_addr[dev];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // pageable sources: each copy returns once the source has been read (it may
    // first wait for the stream's earlier work), so the host tables can be
    // refilled by the next call
    if (ni > 0) e = cudaMemcpyAsync(base + kOffItems, g_items, sizeof(PoItem) * (size_t)ni, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffOff, g_angles, sizeof(PoAngle) * (size_t)n_angles, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffFreq, g_freq, sizeof(float4) * (size_t)n_freq, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffKf, g_kf, sizeof(double) * (size_t)n_freq, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return reject(SBR_ERR_CUDA, "sbr_po_integrate_noalloc: copy of the tables failed");

    pa.rec = (const Record*)records;
    pa.items = (const PoItem*)(base + kOffItems);
    pa.n_items = ni;
    pa.freq = (const float4*)(base + kOffFreq);
    pa.kfreq = (const double*)(base + kOffKf);
    pa.n_freq = (int)n_freq;
    pa.partial = (double*)(base + kOffPartial);  // every entry read below is written by this call first
    e = launch_po(pa, st);
    if (e == cudaSuccess)
        e = launch_po_final(pa.partial, pa.items, (const PoAngle*)(base + kOffOff), (int)n_angles, pa.kfreq, pa.n_pol,
                            E_re_im, rcs_dbsm, st);
    if (e != cudaSuccess) return reject(SBR_ERR_CUDA, "sbr_po_integrate_noalloc: kernel launch failed");
    return SBR_OK;
}

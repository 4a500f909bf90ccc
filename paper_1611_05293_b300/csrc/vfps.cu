// vfps.cu -- runtime and C ABI of the B300 VFP phase-space stepper.
//
// Host side: parameter checks, one device allocation per simulation carved
// into its buffers, the impedance table (FP64 on the host, once per
// vfps_set_impedance), launch groups (instances that share precision,
// interpolation order and CTA width advance in one launch per step), CUDA
// graphs of GRAPH_STEPS launches for long runs, the CSR-power ring drain,
// and the batch/slot bookkeeping.  The per-step work runs in the kernels of
// vfps_kernels.cuh; nothing of the step is computed on the host.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <mutex>
#include <vector>

#include "../../include/vfps.h"
#include "vfps_kernels.cuh"
#include "vfps_fast.cuh"
#include "vfps_pair.cuh"
#include "vfps_haissinski.cuh"

namespace vfps {
void impedance_table(int model, int M, double delta, double Pi, std::vector<std::complex<double>>& z);
}

using namespace vfps;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRingDefault = 1 << 15;  // CSR-power ring entries per simulation
constexpr int kGraphSteps = 32;        // launches per captured CUDA graph
constexpr int kPersistSteps = 256;     // steps per persistent launch (lone simulations)
// polls of a bounded device wait before it gives up with VFPS_ETIMEOUT (each
// poll an acquire load and a short sleep: about a second in all)
constexpr unsigned kSpinLimitDefault = 1u << 21;
constexpr size_t kAlign = 256;
constexpr int kInstanceSlots = 16;     // buffers of one instance's allocation

thread_local char g_last_error[256] = "";

void note_cuda_error(cudaError_t e, const char* where)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

#define CU(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            note_cuda_error(e_, #call);            \
            return VFPS_ECUDA;                     \
        }                                          \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }


int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

int check_params(const vfps_params* p)
{
    if (!p) return VFPS_EINVAL;
    if (p->n < 8 || p->n > 2048) return VFPS_EINVAL;
    if (p->steps_per_period < 2) return VFPS_EINVAL;
    if (p->interp_points < 2 || p->interp_points > 4) return VFPS_EINVAL;
    if (p->clamp != 0 && p->clamp != 1) return VFPS_EINVAL;
    if (p->fp_derivative != 0 && p->fp_derivative != 1) return VFPS_EINVAL;
    if (p->precision != 0 && p->precision != 1) return VFPS_EINVAL;
    if (p->renormalize != 0 && p->renormalize != 1) return VFPS_EINVAL;
    if (p->rotation != 0 && p->rotation != 1) return VFPS_EINVAL;
    if (!(p->half_width > 0.0) || !std::isfinite(p->half_width)) return VFPS_EINVAL;
    if (!(p->beta >= 0.0) || !std::isfinite(p->beta)) return VFPS_EINVAL;
    if (p->pad_factor < 2 || p->pad_factor > 64) return VFPS_EINVAL;
    if ((long long)p->pad_factor * p->n > 16384) return VFPS_EINVAL;
    return VFPS_OK;
}

// FFT length: the smallest power of two >= pad_factor * n.
int fft_length(const vfps_params* p)
{
    int m = 1;
    while (m < p->pad_factor * p->n) m <<= 1;
    return m;
}

// Column halo of the staged slab: 2 nodes of the cubic stencil plus the
// largest source displacement c (|cos phi - 1| + |sin phi|), plus one.
int halo_for(const vfps_params* p)
{
    double phi = 2.0 * kPi / p->steps_per_period;
    double c = 0.5 * (p->n - 1);
    double cm1 = std::fabs(-2.0 * std::sin(0.5 * phi) * std::sin(0.5 * phi));
    double dmax = c * (cm1 + std::fabs(std::sin(phi)));
    // Manhattan drift: row y moves by h (y - c), h = 2 sin(phi/2)
    dmax = std::max(dmax, c * 2.0 * std::fabs(std::sin(0.5 * phi)));
    return 3 + (int)std::ceil(dmax);
}

int elem_size(const vfps_params* p) { return p->precision ? 8 : 4; }

size_t step_smem(const vfps_params* p, int W)
{
    size_t es = elem_size(p);
    int h = halo_for(p);
    size_t slab = (size_t)(W + 2 * h) * (p->n + 4) * es;
    size_t cols = (size_t)W * p->n * es;
    size_t fin = vfps::finalise_smem(fft_length(p), p->n, W * 32, 2 * (int)es);
    return align_up(std::max(slab + cols, fin), 16);
}

int g_max_smem = -1;

// Device allocations of the library go through here.  VFPS_FAULT_ALLOC=k in
// the environment makes the k-th allocation of the process (1-based) fail
// with ENOMEM without touching the device -- the host-side fault injection
// the error-path tests use; the allocations after it succeed again.
long long g_alloc_count = 0;

cudaError_t dev_alloc(void** ptr, size_t bytes)
{
    static const long long fail_at = [] {
        const char* e = std::getenv("VFPS_FAULT_ALLOC");
        return e ? std::atoll(e) : 0LL;
    }();
    if (fail_at > 0 && ++g_alloc_count == fail_at) return cudaErrorMemoryAllocation;
    return cudaMalloc(ptr, bytes);
}

// NVTX range for the duration of a scope (host-side trace of the API calls).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int device_smem_limit()
{
    if (g_max_smem < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
        g_max_smem = v;
    }
    return g_max_smem;
}

// The FP32 register-blocked kernel (vfps_fast.cuh) covers cubic
// interpolation without clamping on grids with n a multiple of 4, for both
// rotations.
bool fast_eligible(const vfps_params* p)
{
    // the Manhattan drift's x-node may step by at most one per 4-row block:
    // h = 2 sin(pi/steps) < 1/3
    return p->precision == 0 && p->interp_points >= 2 && p->interp_points <= 4 && (p->n % 4) == 0 &&
           (p->rotation == 0 || p->steps_per_period >= 20);
}

// Rows per lane of the FP32 kernel's kick/FP blocks: 8 where n allows.
int fast_kr(int n) { return (n % 8 == 0) ? 8 : 4; }

size_t fast_smem(const vfps_params* p, int W)
{
    size_t fin = vfps::finalise_smem(fft_length(p), p->n, W * 32, 8);
    return align_up(std::max(vfps::fast_ring_smem(p->n, halo_for(p), W, p->rotation == 1), fin), 16);
}

// The pair kernel (vfps_pair.cuh) covers what the FP32 register-blocked
// kernel covers for the standard rotation, on grids with n a multiple of 32
// (rows per lane of its copies) and a column halo of at most 12 (its windows
// then stay inside the kPairRP padding pair-rows of a ring column).
bool pair_eligible(const vfps_params* p)
{
    return fast_eligible(p) && p->interp_points == 4 && !p->clamp && p->rotation == 0 && (p->n % 32) == 0 &&
           p->n < 512 && halo_for(p) <= 12;
}

size_t pair_smem(const vfps_params* p, int W)
{
    size_t fin = vfps::finalise_smem(fft_length(p), p->n, W * 32, 8);
    return align_up(std::max(vfps::pair_ring_smem(p->n, halo_for(p), W), fin), 16);
}

int g_num_sms = 0;

int num_sms()
{
    if (g_num_sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            g_num_sms = 1;
    }
    return g_num_sms;
}

int g_smem_per_sm = -1;

int device_smem_per_sm()
{
    if (g_smem_per_sm < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
        g_smem_per_sm = v;
    }
    return g_smem_per_sm;
}

// CTA width in columns (8, 4 or 2) for one kernel: 0 if none fits.  The
// kernels also use a few bytes of static shared memory; keep 1 KB for it.
// Batches take the widest width that fits: fewest CTAs and the least halo
// re-read per column.  With latency set (one simulation on its own) a step
// lasts as long as its slowest CTA plus the finaliser that the last CTA
// runs with W x 32 threads: the widest width is taken whose grid still has
// at least 0.4 x SMs CTAs (measured per step: N = 256 at W = 2 / 4 / 8 10.8 /
// 10.2 / 10.8 us, N = 1024 at W = 4 / 8 20.5 / 19.5 us); for grids too small
// for that, the narrowest whose CTAs all fit on the device at once (one wave:
// ceil(n/W) <= SMs x CTAs per SM, limited by shared memory and 32 per SM).
int pick_width(const vfps_params* p, bool fast, bool latency)
{
    const long long lim = device_smem_limit() - 1024;
    const int widths[3] = {8, 4, 2};
    int best = 0, wide = 0, four = 0;
    for (int W : widths) {
        const long long need = (long long)(fast ? fast_smem(p, W) : step_smem(p, W));
        if (need > lim) continue;
        if (!best) best = W;
        if (W == 4) four = 4;
        if (latency) {
            const long long ctas = (p->n + W - 1) / W;
            const long long per_sm = std::min<long long>(32, device_smem_per_sm() / (need + 1024));
            // FP32 kernel: never the 2-wide CTA for a lone simulation, whose
            // last CTA then finalises with one transform warp (measured
            // slower at every n from 48 to 384)
            if (!wide && 5 * ctas >= 2LL * num_sms() && (!fast || W >= 4)) wide = W;
            if (ctas <= (long long)num_sms() * per_sm) best = W;
        }
    }
    if (latency && fast && !wide && four) wide = four;
    return (latency && wide) ? wide : best;
}

// *fast is set when the FP32 register-blocked kernel applies and fits.
int choose_width(const vfps_params* p, int* fast = nullptr, bool latency = false)
{
    if (fast) *fast = 0;
    if (fast_eligible(p)) {
        // N_I = 2, 3 and clamping have one FP32-kernel width, W = 4
        const int W = (p->interp_points == 4 && !p->clamp) ? pick_width(p, true, latency)
                      : ((long long)fast_smem(p, 4) <= device_smem_limit() - 1024 ? 4 : 0);
        if (W) {
            if (fast) *fast = 1;
            return W;
        }
    }
    return pick_width(p, false, latency);
}

// ----------------------------------------------------------------------------
// One simulation: a single device allocation holding every buffer.
struct Instance {
    vfps_params p{};
    int n = 0, ld = 0, M = 0, W = 0, ntiles = 0, ring = kRingDefault;
    int fast = 0;  // 1: FP32 register-blocked step kernel
    double delta = 0, phi = 0;
    int model = 0;
    double Pi = 0, S = 0;
    void* dmem = nullptr;
    size_t dbytes = 0;
    std::shared_ptr<void> arena;  // set when dmem lies in a block shared with other slots
    void* psi[2] = {nullptr, nullptr};
    void* zhat = nullptr;
    void* tw = nullptr;
    double* colsum = nullptr;
    double* rho = nullptr;
    void* kick = nullptr;
    void* kickw = nullptr;   // FP32: two float4 per column
    double* mom = nullptr;   // moments scratch: 3n column sums, then the 4 results
    // persistent launches: tagged column-sum words, tagged kick records, step flags
    unsigned long long* cword = nullptr;
    unsigned long long* rword = nullptr;
    unsigned long long* sword = nullptr;
    unsigned* cflag = nullptr;
    double* pring = nullptr;
    double* qring = nullptr;
    DevState* st = nullptr;
    unsigned char hdesc[sizeof(Desc<double>)];  // host copy of the descriptor
    void* ddesc = nullptr;                       // device copy
    int2* dtiles = nullptr;                      // this instance alone: its tiles
    int4* dsegs = nullptr;                       // ... and one FP32-kernel segment per tile
    // host bookkeeping
    long long steps_queued = 0;   // steps launched so far
    long long drained = 0;        // ring entries already moved to the host
    long long target = -1;        // batch slots: total steps wanted
    int parity0 = 0;
    std::vector<double> pw, qw;   // drained series
    size_t pw_taken = 0, qw_taken = 0;
    // moments recorded by the step's epilogue (vfps_record_moments)
    int mom_every = 0;            // 0: off
    double* mring = nullptr;      // ring entries x 4 doubles, allocated on first use
    long long mdrained = 0;       // states t <= mdrained are on the host (or not recorded)
    std::vector<double> mw;       // drained records: t, <q>, sigma_q, <p>, sigma_p
    size_t mw_taken = 0;
    // bounded waits of persistent launches (vfps_create reads both from the
    // environment: VFPS_SPIN_LIMIT, and the test hook VFPS_FAULT_NO_SIGNAL)
    unsigned spin_limit = kSpinLimitDefault;
    int fault_no_signal = 0;
};

// Persistent launches: tagged 64-bit words (2n column-sum halves, n kick
// records, a scale per worker CTA -- at most n/2 + 1 of them), then a step
// flag per worker CTA.
size_t persist_bytes(int n) { return (size_t)(2 * n + n / 2 + 2) * 8 + (size_t)(n + 2) * 4; }

size_t instance_bytes(const vfps_params* p, int ring, size_t* offs)
{
    size_t es = elem_size(p);
    int n = p->n;
    int ld = (int)align_up(n, 16 / es);
    int M = fft_length(p);
    size_t o = 0;
    auto take = [&](int slot, size_t b) {
        o = align_up(o, kAlign);
        offs[slot] = o;
        o += b;
    };
    take(0, (size_t)n * ld * es);        // psi0
    take(1, (size_t)n * ld * es);        // psi1
    take(2, (size_t)(M / 2 + 1) * 2 * es);  // zhat
    take(3, (size_t)(M / 2) * 2 * es);   // twiddles
    take(4, (size_t)n * 8);              // colsum
    take(5, (size_t)n * 8);              // rho
    take(6, (size_t)n * es);             // kick
    take(7, (size_t)ring * 8);           // pring
    take(8, (size_t)ring * 8);           // qring
    take(9, sizeof(DevState));           // state
    take(10, sizeof(Desc<double>));      // descriptor
    take(11, sizeof(int2) * (size_t)((n + 1) / 2 + 1));  // tiles (W >= 2)
    take(12, (size_t)n * 32);            // kick table (FP32 path)
    take(13, (size_t)(3 * n + 4) * 8);   // moments scratch
    take(14, sizeof(int4) * (size_t)((n + 1) / 2 + 1));  // FP32-kernel segments (W >= 2)
    take(15, persist_bytes(n));          // persistent launches: tagged words, step flags
    return align_up(o, kAlign);
}

template <typename T>
void fill_desc(Instance& I)
{
    Desc<T> d{};
    d.psi[0] = (T*)I.psi[0];
    d.psi[1] = (T*)I.psi[1];
    d.zhat = (const typename C2<T>::type*)I.zhat;
    d.tw = (const typename C2<T>::type*)I.tw;
    d.colsum = I.colsum;
    d.rho = I.rho;
    d.kick = (T*)I.kick;
    d.kickw = (float4*)I.kickw;
    d.pring = I.pring;
    d.qring = I.qring;
    d.mring = I.mring;
    d.colmom = I.mom;  // the moments scratch (3n + 4 doubles) holds the 2n column sums
    d.cword = I.cword;
    d.rword = I.rword;
    d.sword = I.sword;
    d.cflag = I.cflag;
    d.mom_every = I.mring ? I.mom_every : 0;
    d.ni = I.p.interp_points;
    d.spin_limit = I.spin_limit;
    d.fault_no_signal = I.fault_no_signal;
    d.st = I.st;
    d.n = I.n;
    d.ld = I.ld;
    d.M = I.M;
    d.logM = ilog2(I.M);
    d.ring_mask = I.ring - 1;
    d.renorm = I.p.renormalize;
    d.clamp = I.p.clamp;
    d.h = halo_for(&I.p);
    d.ntiles = I.ntiles;
    d.rotation = I.p.rotation;
    d.hm = T(2.0 * std::sin(kPi / I.p.steps_per_period));
    double phi = I.phi;
    double s2 = std::sin(0.5 * phi);
    d.cm1 = T(-2.0 * s2 * s2);
    d.sn = T(std::sin(phi));
    d.c = T(0.5 * (I.n - 1));
    // FP increment g_k(y) psi_b(y+k), k = -1..2:  h (a_k + b_k p_y), p_y = -L + y Delta
    double hh = I.p.beta / I.p.steps_per_period, D = I.delta, L = I.p.half_width;
    double a[4], b[4];
    a[0] = 1.0 / (D * D); a[1] = 1.0 - 2.0 / (D * D); a[2] = 1.0 / (D * D); a[3] = 0.0;
    if (I.p.fp_derivative) {  // Eq. cubic diff: (-2 f_{-1} - 3 f_0 + 6 f_1 - f_2) / (6 Delta)
        b[0] = -2.0 / (6.0 * D); b[1] = -3.0 / (6.0 * D); b[2] = 6.0 / (6.0 * D); b[3] = -1.0 / (6.0 * D);
    } else {                  // central: (f_1 - f_{-1}) / (2 Delta)
        b[0] = -1.0 / (2.0 * D); b[1] = 0.0; b[2] = 1.0 / (2.0 * D); b[3] = 0.0;
    }
    for (int k = 0; k < 4; ++k) {
        d.ga[k] = T(hh * (a[k] - b[k] * L));
        d.gb[k] = T(hh * b[k] * D);
    }
    d.delta = I.delta;
    d.dkappa = 2.0 * kPi / (I.M * I.delta);
    d.kick_per_v = I.S * I.phi / I.delta;
    std::memcpy(I.hdesc, &d, sizeof(d));
}

int upload_desc(Instance& I, cudaStream_t s)
{
    if (I.p.precision) fill_desc<double>(I);
    else fill_desc<float>(I);
    CU(cudaMemcpyAsync(I.ddesc, I.hdesc, sizeof(Desc<double>), cudaMemcpyHostToDevice, s));
    return VFPS_OK;
}

void destroy_instance(Instance* I)
{
    if (!I) return;
    if (I->mring) cudaFree(I->mring);
    if (I->dmem && !I->arena) cudaFree(I->dmem);  // a shared block goes with its last slot
    delete I;
}

// Pinned host staging for the state, status and series copies, one per host
// thread (a thread's calls are sequential; threads do not share one), grown
// to the largest transfer and released when the thread ends.  Pinned copies
// skip the driver's pageable bounce buffer, and a buffer kept for the
// thread's life takes no page faults.  Every user finishes with the staged
// data (after a stream synchronisation) before it returns.
struct HostStage {
    unsigned char* p = nullptr;
    size_t cap = 0;
    unsigned char* get(size_t bytes)
    {
        if (bytes <= cap) return p;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max(bytes, (size_t)1 << 20);
        if (cudaHostAlloc((void**)&p, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return nullptr;
        }
        cap = want;
        return p;
    }
    ~HostStage()
    {
        if (p) cudaFreeHost(p);
    }
};

HostStage& host_stage()
{
    thread_local HostStage st;
    return st;
}

// Staged layout of a state transfer: the status word, then the psi buffer.
constexpr size_t kStageHead = 256;

// Unit Gaussian exp(-(q^2+p^2)/2) on an instance's grid (the default start).
void unit_gaussian(const Instance& I, double* g)
{
    const int n = I.n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double q = -I.p.half_width + i * I.delta, pp = -I.p.half_width + j * I.delta;
            g[(size_t)i * n + j] = std::exp(-0.5 * (q * q + pp * pp));
        }
}

// CTAs per state of the staging kernels (one row or more each): about four
// per SM over the whole transfer, at least 4 per state and at most n.
int stage_rows(int n, int count)
{
    const int want = 4 * num_sms() / std::max(1, count);
    return std::min(n, std::max(4, want));
}

// Host states -> normalised device states of `count` instances of one
// precision: one copy of all of them to the device, FP64 charge sums there
// (stage_sum_kernel), a check that every value is finite and every charge
// positive, then psi[parity] = psi * 1/(Delta^2 sum) in the instance's type
// with a pending scale of 1 (stage_store_kernel).  src: the states back to
// back (n*n doubles each) or null for unit Gaussians.  Interpolation
// overshoots leave small negative densities in evolved states (Sec. IV.B), so
// only non-finite values and a non-positive total charge are refused
// (EINVAL, before anything is stored).  Synchronises s.
template <typename T>
int upload_states_t(Instance* const* inst, int count, const double* src, cudaStream_t s)
{
    std::vector<long long> off((size_t)count);
    long long total = 0;
    for (int i = 0; i < count; ++i) {
        off[(size_t)i] = total;
        total += (long long)inst[i]->n * inst[i]->n;
    }
    std::vector<double> gauss;
    if (!src) {
        gauss.resize((size_t)total);
        for (int i = 0; i < count; ++i) unit_gaussian(*inst[i], gauss.data() + off[(size_t)i]);
        src = gauss.data();
    }
    const size_t vb = align_up((size_t)total * 8, kAlign), sb = align_up((size_t)count * 16, kAlign);
    const size_t pb = align_up((size_t)count * 16 * kStageParts, kAlign);
    const size_t jb = sizeof(StateJob<T>) * (size_t)count;
    std::vector<StateJob<T>> jobs((size_t)count);
    for (int i = 0; i < count; ++i) {
        const Instance& I = *inst[i];
        jobs[(size_t)i] = StateJob<T>{{(T*)I.psi[0], (T*)I.psi[1]}, I.st, off[(size_t)i], I.delta * I.delta, I.n, I.ld};
    }
    unsigned char* d = nullptr;
    CU(cudaMallocAsync((void**)&d, vb + sb + pb + jb, s));
    double* dv = (double*)d;
    double* ds = (double*)(d + vb);
    double* dp = (double*)(d + vb + sb);
    StateJob<T>* dj = (StateJob<T>*)(d + vb + sb + pb);
    std::vector<double> sums((size_t)count * 2);
    cudaError_t e = cudaMemcpyAsync(dv, src, (size_t)total * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dj, jobs.data(), jb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        stage_sum_kernel<<<dim3(kStageParts, (unsigned)count), 256, 0, s>>>(dv, (long long)inst[0]->n * inst[0]->n,
                                                                            dp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        stage_combine_kernel<<<(count + 255) / 256, 256, 0, s>>>(dp, count, ds);
        e = cudaGetLastError();
    }
    // (one grid size per call: stage_sum_kernel strides by the first state's size)
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums.data(), ds, sums.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = VFPS_OK;
    if (e != cudaSuccess) {
        note_cuda_error(e, "state upload");
        rc = VFPS_ECUDA;
    }
    for (int i = 0; i < count && rc == VFPS_OK; ++i)
        if (!(sums[2 * (size_t)i + 1] == 1.0) || !(sums[2 * (size_t)i] > 0.0)) rc = VFPS_EINVAL;
    if (rc == VFPS_OK) {
        const int rows = stage_rows(inst[0]->n, count);
        stage_store_kernel<T><<<dim3((unsigned)rows, (unsigned)count), 256, 0, s>>>(dv, ds, dj);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            note_cuda_error(e, "state upload");
            rc = VFPS_ECUDA;
        }
    }
    cudaFreeAsync(d, s);
    return rc;
}

int upload_states(Instance* const* inst, int count, const double* src, cudaStream_t s)
{
    if (count < 1) return VFPS_OK;
    for (int i = 1; i < count; ++i)
        if (inst[i]->p.precision != inst[0]->p.precision || inst[i]->n != inst[0]->n) return VFPS_EINVAL;
    return inst[0]->p.precision ? upload_states_t<double>(inst, count, src, s)
                                : upload_states_t<float>(inst, count, src, s);
}

// psi (host, n*n doubles, or null for the unit Gaussian) -> normalised device
// psi[parity]; the pending scale is 1.
int upload_psi(Instance& I, const double* psi, cudaStream_t s)
{
    Instance* p = &I;
    return upload_states(&p, 1, psi, s);
}

// Tables are costly for the shielded model (an Airy sum per frequency), and a
// parameter scan reuses a few (model, M, Delta, Pi): keep the last 64.
void cached_impedance(int model, int M, double delta, double Pi, std::vector<std::complex<double>>& z)
{
    static std::mutex mu;  // handles and batches may be driven from several threads
    std::lock_guard<std::mutex> lk(mu);
    static std::map<std::tuple<int, int, double, double>, std::vector<std::complex<double>>> cache;
    static std::deque<std::tuple<int, int, double, double>> order;
    auto key = std::make_tuple(model, M, delta, model == 2 ? Pi : 0.0);
    auto it = cache.find(key);
    if (it != cache.end()) {
        z = it->second;
        return;
    }
    vfps::impedance_table(model, M, delta, Pi, z);
    cache[key] = z;
    order.push_back(key);
    if (order.size() > 64) {
        cache.erase(order.front());
        order.pop_front();
    }
}

// The instance's impedance table for a model in its element type (buf), and
// the model, Pi and S_csr recorded in the instance.  Errors: EINVAL.
int impedance_image(Instance& I, int model, double Pi, double S, const double* table, std::vector<unsigned char>& buf)
{
    int K = I.M / 2;
    std::vector<std::complex<double>> z;
    if (model == VFPS_IMPEDANCE_TABLE) {
        if (!table) return VFPS_EINVAL;
        z.resize(K + 1);
        for (int k = 0; k <= K; ++k) {
            z[k] = {table[2 * k], table[2 * k + 1]};
            if (!std::isfinite(z[k].real()) || !std::isfinite(z[k].imag())) return VFPS_EINVAL;
        }
    } else if (model >= 0 && model <= 2) {
        if (model == 2 && !(Pi > 0.0)) return VFPS_EINVAL;
        cached_impedance(model, I.M, I.delta, Pi, z);
    } else {
        return VFPS_EINVAL;
    }
    if (!std::isfinite(S)) return VFPS_EINVAL;
    size_t es = elem_size(&I.p);
    buf.resize((size_t)(K + 1) * 2 * es);
    for (int k = 0; k <= K; ++k) {
        if (es == 8) {
            reinterpret_cast<double*>(buf.data())[2 * k] = z[k].real();
            reinterpret_cast<double*>(buf.data())[2 * k + 1] = z[k].imag();
        } else {
            reinterpret_cast<float*>(buf.data())[2 * k] = (float)z[k].real();
            reinterpret_cast<float*>(buf.data())[2 * k + 1] = (float)z[k].imag();
        }
    }
    I.model = model;
    I.Pi = Pi;
    I.S = S;
    return VFPS_OK;
}

int upload_impedance(Instance& I, int model, double Pi, double S, const double* table, cudaStream_t s)
{
    std::vector<unsigned char> buf;
    const int rc = impedance_image(I, model, Pi, S, table, buf);
    if (rc) return rc;
    CU(cudaMemcpyAsync(I.zhat, buf.data(), buf.size(), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    return VFPS_OK;
}

// An instance's buffers inside its one allocation b (offsets of instance_bytes).
void set_pointers(Instance& I, unsigned char* b, const size_t* offs)
{
    I.psi[0] = b + offs[0];
    I.psi[1] = b + offs[1];
    I.zhat = b + offs[2];
    I.tw = b + offs[3];
    I.colsum = (double*)(b + offs[4]);
    I.rho = (double*)(b + offs[5]);
    I.kick = b + offs[6];
    I.pring = (double*)(b + offs[7]);
    I.qring = (double*)(b + offs[8]);
    I.st = (DevState*)(b + offs[9]);
    I.ddesc = b + offs[10];
    I.dtiles = (int2*)(b + offs[11]);
    I.kickw = b + offs[12];
    I.mom = (double*)(b + offs[13]);
    I.dsegs = (int4*)(b + offs[14]);
    I.cword = (unsigned long long*)(b + offs[15]);
    I.rword = I.cword + (size_t)I.n;
    I.sword = I.rword + (size_t)I.n;
    I.cflag = reinterpret_cast<unsigned*>(I.sword + (size_t)I.n / 2 + 2);
}

// Host images of an instance's constant tables, in its own element type:
// twiddles exp(-2 pi i k/M) (FP64 on the host), and the impedance table of a
// model (FP64 host table, rounded once).
void twiddle_table(const Instance& I, std::vector<unsigned char>& buf)
{
    const int K = I.M / 2;
    const size_t es = elem_size(&I.p);
    buf.resize((size_t)K * 2 * es);
    for (int k = 0; k < K; ++k) {
        const double ang = -2.0 * kPi * k / I.M;
        const double c = std::cos(ang), s = std::sin(ang);
        if (es == 8) {
            reinterpret_cast<double*>(buf.data())[2 * k] = c;
            reinterpret_cast<double*>(buf.data())[2 * k + 1] = s;
        } else {
            reinterpret_cast<float*>(buf.data())[2 * k] = (float)c;
            reinterpret_cast<float*>(buf.data())[2 * k + 1] = (float)s;
        }
    }
}

int create_instance(const vfps_params* p, const double* psi0, int ring, cudaStream_t s, Instance** out,
                    bool latency = false, bool upload = true, bool tables = true,
                    std::shared_ptr<void> arena = nullptr, size_t arena_off = 0)
{
    int rc = check_params(p);
    if (rc) return rc;
    int fast = 0;
    int W = choose_width(p, &fast, latency);
    if (W == 0) return VFPS_EINVAL;  // grid too large for the staged slab at this step angle
    std::unique_ptr<Instance, void (*)(Instance*)> I(new (std::nothrow) Instance(), destroy_instance);
    if (!I) return VFPS_ENOMEM;
    I->p = *p;
    I->n = p->n;
    I->ld = (int)align_up(p->n, 16 / elem_size(p));
    I->M = fft_length(p);
    I->W = W;
    I->fast = fast;
    I->ntiles = (p->n + W - 1) / W;
    I->ring = ring;
    I->delta = 2.0 * p->half_width / (p->n - 1);
    I->phi = 2.0 * kPi / p->steps_per_period;
    size_t offs[kInstanceSlots];
    I->dbytes = instance_bytes(p, ring, offs);
    if (arena) {  // a slice of a block the caller allocated and cleared
        I->arena = arena;
        I->dmem = (unsigned char*)arena.get() + arena_off;
    } else {
        if (dev_alloc(&I->dmem, I->dbytes) != cudaSuccess) {
            cudaGetLastError();
            return VFPS_ENOMEM;
        }
        if (cudaMemsetAsync(I->dmem, 0, I->dbytes, s) != cudaSuccess) return VFPS_ECUDA;
    }
    unsigned char* b = (unsigned char*)I->dmem;
    set_pointers(*I, b, offs);
    if (!tables) {  // the caller uploads every table (vfps_batch_add_many)
        *out = I.release();
        return VFPS_OK;
    }
    // twiddles exp(-2 pi i k/M), FP64 on the host
    {
        std::vector<unsigned char> buf;
        twiddle_table(*I, buf);
        // a copy from pageable memory returns once the data is staged: buf may go
        if (cudaMemcpyAsync(I->tw, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return VFPS_ECUDA;
    }
    {
        std::vector<int2> t(I->ntiles);
        std::vector<int4> sg(I->ntiles);
        for (int i = 0; i < I->ntiles; ++i) {
            t[i] = make_int2(0, i * W);
            sg[i] = make_int4(0, i * W, 1, 0);
        }
        if (cudaMemcpyAsync(I->dtiles, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(I->dsegs, sg.data(), sizeof(int4) * sg.size(), cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
            return VFPS_ECUDA;
        DevState st{};
        st.scale = 1.0;
        if (cudaMemcpyAsync(I->st, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess) return VFPS_ECUDA;
    }
    rc = upload_impedance(*I, 0, 0.0, 0.0, nullptr, s);
    if (rc) return rc;
    if (upload) {
        rc = upload_psi(*I, psi0, s);
        if (rc) return rc;
    }
    *out = I.release();
    return VFPS_OK;
}

// ----------------------------------------------------------------------------
// Launch groups: instances with equal (precision, N_I, W) advance in one
// launch per step.  The tile table lists (instance, first column) per CTA.
struct Group {
    int prec = 0, ni = 4, W = 8, fast = 0;
    int var = 0;  // FP32 kernel instance: 0 cubic, 1 N_I = 2 or 3 (from the descriptor), 2 clamped
    int tps = 1;  // FP32 streaming kernel: consecutive tiles per CTA
    int kr = 4;   // FP32 streaming kernel: rows per lane of the kick/FP blocks
    int n = 0;    // grid size shared by the group's instances
    int rot = 0;  // rotation shared by the group's instances (FP32 streaming kernel)
    int pair = 0; // 1: members 2k, 2k+1 advance together in the pair kernel
    // batches: members, where their descriptors and tiles sit in the batch
    // arrays, and the autotuner's state (candidates (W, tps) still to time)
    std::vector<Instance*> members;
    size_t off_d = 0, off_t = 0;
    std::vector<std::pair<int, int>> cands;
    std::vector<float> cand_ms;
    int cand = -1;  // candidate of the step in flight; -1 = warm-up step
    std::tuple<int, int, int, int, int, int> tune_key;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    size_t smem = 0;
    int ntiles = 0;
    void* ddescs = nullptr;  // array of Desc<T>
    int2* dtiles = nullptr;
    int4* dsegs = nullptr;   // FP32 kernels: spc segments per CTA, grid CTAs
    int spc = 1, grid = 0;
    size_t seg_cap = 0;      // batch groups: room for segments (entries)
    size_t tab_bytes = 0;    // batch groups: bytes of descriptors + tile/segment table
    double share = 1.0;      // batch groups: fraction of the batch's FP32 cells in this group
    cudaStream_t stream = nullptr;  // batch groups: their own (forked) stream
};

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream finishes; it waits (griddepcontrol.wait)
// before reading anything that kernel produced.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename T, int NI, int W>
int launch_step_t(const Group& g, cudaStream_t s)
{
    CU(launch_pdl(step_kernel<T, NI, W>, g.ntiles, W * 32, g.smem, s, (const Desc<T>*)g.ddescs,
                  (const int2*)g.dtiles));
    return VFPS_OK;
}

template <typename T, int W>
int launch_project_t(const Group& g, cudaStream_t s)
{
    CU(launch_pdl(project_kernel<T, W>, g.ntiles, W * 32, g.smem, s, (const Desc<T>*)g.ddescs,
                  (const int2*)g.dtiles));
    return VFPS_OK;
}

template <typename T, int NI>
int launch_step_w(const Group& g, cudaStream_t s)
{
    switch (g.W) {
    case 8: return launch_step_t<T, NI, 8>(g, s);
    case 4: return launch_step_t<T, NI, 4>(g, s);
    case 2: return launch_step_t<T, NI, 2>(g, s);
    }
    return VFPS_EINVAL;
}

template <typename T>
int launch_step_ni(const Group& g, cudaStream_t s)
{
    switch (g.ni) {
    case 4: return launch_step_w<T, 4>(g, s);
    case 3: return launch_step_w<T, 3>(g, s);
    case 2: return launch_step_w<T, 2>(g, s);
    }
    return VFPS_EINVAL;
}

template <int W, int KR, int NC, int NI = 4>
int launch_fast_k(const Group& g, cudaStream_t s)
{
    if (g.rot)
        CU(launch_pdl(step_kernel_f32<W, KR, NC, 1, NI>, g.grid, fast_threads(W, NC), g.smem, s,
                      (const Desc<float>*)g.ddescs, (const int4*)g.dsegs, g.spc));
    else
        CU(launch_pdl(step_kernel_f32<W, KR, NC, 0, NI>, g.grid, fast_threads(W, NC), g.smem, s,
                      (const Desc<float>*)g.ddescs, (const int4*)g.dsegs, g.spc));
    return VFPS_OK;
}

template <int W, int NC>
int launch_pair_k(const Group& g, cudaStream_t s)
{
    CU(launch_pdl(step_kernel_f32x2<W, NC>, g.grid, W * 32, g.smem, s, (const Desc<float>*)g.ddescs,
                  (const int4*)g.dsegs, g.spc));
    return VFPS_OK;
}

template <int W>
int launch_pair_t(const Group& g, cudaStream_t s)
{
    if (g.n == 256) return launch_pair_k<W, 256>(g, s);
    if (g.n == 1024) return launch_pair_k<W, 1024>(g, s);
    return launch_pair_k<W, 0>(g, s);
}

// The hot grid sizes (N = 256 scans, N = 1024 single runs) have their own
// compiled instances with n fixed at compile time.
template <int W>
int launch_fast_t(const Group& g, cudaStream_t s)
{
    if (g.var) {  // N_I = 2, 3 (NI = 0) or clamping (NI = 1): W = 4 only
        if constexpr (W == 4) {
            if (g.var == 2) return g.kr == 8 ? launch_fast_k<4, 8, 0, 1>(g, s) : launch_fast_k<4, 4, 0, 1>(g, s);
            return g.kr == 8 ? launch_fast_k<4, 8, 0, 0>(g, s) : launch_fast_k<4, 4, 0, 0>(g, s);
        }
        return VFPS_EINVAL;
    }
    if (g.kr == 8) {
        if (g.n == 256) return launch_fast_k<W, 8, 256>(g, s);
        if (g.n == 1024) return launch_fast_k<W, 8, 1024>(g, s);
        if (g.n == 512) return launch_fast_k<W, 8, 512>(g, s);
        return launch_fast_k<W, 8, 0>(g, s);
    }
    return launch_fast_k<W, 4, 0>(g, s);
}

int launch_step(const Group& g, cudaStream_t s)
{
    if (g.ntiles == 0) return VFPS_OK;
    if (g.pair) {
        switch (g.W) {
        case 8: return launch_pair_t<8>(g, s);
        case 4: return launch_pair_t<4>(g, s);
        case 2: return launch_pair_t<2>(g, s);
        }
        return VFPS_EINVAL;
    }
    if (g.fast) {
        switch (g.W) {
        case 8: return launch_fast_t<8>(g, s);
        case 4: return launch_fast_t<4>(g, s);
        case 2: return launch_fast_t<2>(g, s);
        }
        return VFPS_EINVAL;
    }
    return g.prec ? launch_step_ni<double>(g, s) : launch_step_ni<float>(g, s);
}

int launch_project(const Group& g, cudaStream_t s)
{
    if (g.ntiles == 0) return VFPS_OK;
    if (g.prec) {
        switch (g.W) {
        case 8: return launch_project_t<double, 8>(g, s);
        case 4: return launch_project_t<double, 4>(g, s);
        case 2: return launch_project_t<double, 2>(g, s);
        }
    } else {
        switch (g.W) {
        case 8: return launch_project_t<float, 8>(g, s);
        case 4: return launch_project_t<float, 4>(g, s);
        case 2: return launch_project_t<float, 2>(g, s);
        }
    }
    return VFPS_EINVAL;
}

// Persistent launches of one lone FP32 simulation (step_persistent_f32), at
// the widths a lone simulation takes (4 and 8) and the compiled grid sizes;
// null where there is no such kernel.
template <int W>
const void* persist_fn_w(int kr, int n, int rot)
{
    if (kr == 8) {
        if (n == 256)
            return rot ? (const void*)step_persistent_f32<W, 8, 256, 1> : (const void*)step_persistent_f32<W, 8, 256, 0>;
        if (n == 1024)
            return rot ? (const void*)step_persistent_f32<W, 8, 1024, 1>
                       : (const void*)step_persistent_f32<W, 8, 1024, 0>;
        if (n == 512)
            return rot ? (const void*)step_persistent_f32<W, 8, 512, 1> : (const void*)step_persistent_f32<W, 8, 512, 0>;
        return rot ? (const void*)step_persistent_f32<W, 8, 0, 1> : (const void*)step_persistent_f32<W, 8, 0, 0>;
    }
    return rot ? (const void*)step_persistent_f32<W, 4, 0, 1> : (const void*)step_persistent_f32<W, 4, 0, 0>;
}

const void* persist_fn(const Group& g)
{
    if (!g.fast || g.pair || g.var) return nullptr;
    if (g.W == 8) return persist_fn_w<8>(g.kr, g.n, g.rot);
    if (g.W == 4) return persist_fn_w<4>(g.kr, g.n, g.rot);
    return nullptr;
}

// Threads per CTA of an FP32 group's kernel (the N = 1024 instance has two
// warps per column).
int group_threads(const Group& g)
{
    return g.W * 32 * ((g.fast && !g.pair && !g.var && g.kr == 8 && (g.n == 512 || g.n == 1024)) ? 2 : 1);
}


// K steps of a lone simulation in one cooperative launch: g.grid worker CTAs
// and one finaliser CTA.  First every tagged word and step flag goes to 0
// (a launch's own steps are tagged from 1; a launch that timed out leaves
// them anyhow).
int launch_persistent(const Group& g, const Instance& I, int K, cudaStream_t s)
{
    const void* f = persist_fn(g);
    if (!f || K <= 0 || g.grid > I.n / 2 + 2) return VFPS_EINVAL;
    CU(cudaMemsetAsync(I.cword, 0, persist_bytes(I.n), s));
    const Desc<float>* d = (const Desc<float>*)g.ddescs;
    const int4* sg = (const int4*)g.dsegs;
    void* args[3] = {(void*)&d, (void*)&sg, (void*)&K};
    CU(cudaLaunchCooperativeKernel(f, dim3(g.grid + 1), dim3(group_threads(g)), args, g.smem, s));
    return VFPS_OK;
}

// Allow every kernel variant the device's full opt-in shared memory (once,
// before any launch or stream capture).
template <typename K>
cudaError_t set_smem_attr_one(K kernel, int lim)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                lim - (int)fa.sharedSizeBytes);
}

template <typename T, int NI, int W>
cudaError_t set_smem_attr(int lim)
{
    cudaError_t e = set_smem_attr_one(step_kernel<T, NI, W>, lim);
    if (e != cudaSuccess) return e;
    if (NI == 4) e = set_smem_attr_one(project_kernel<T, W>, lim);
    return e;
}

template <typename T>
cudaError_t set_smem_attr_all(int lim)
{
    cudaError_t e = cudaSuccess;
    cudaError_t r;
#define VFPS_SET(NI, W) if ((r = set_smem_attr<T, NI, W>(lim)) != cudaSuccess) e = r;
    VFPS_SET(4, 8) VFPS_SET(4, 4) VFPS_SET(4, 2)
    VFPS_SET(3, 8) VFPS_SET(3, 4) VFPS_SET(3, 2)
    VFPS_SET(2, 8) VFPS_SET(2, 4) VFPS_SET(2, 2)
#undef VFPS_SET
    return e;
}

int g_kernels_ready = 0;

int init_kernels()
{
    if (g_kernels_ready) return VFPS_OK;
    int lim = device_smem_limit();
    if (lim <= 0) return VFPS_ECUDA;
    CU(set_smem_attr_all<float>(lim));
    CU(set_smem_attr_all<double>(lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 4, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 4, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 256, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 256, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 256, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 1024, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 1024, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 1024, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 512, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 512, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 512, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 4, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 4, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 256, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 256, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 256, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 1024, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 1024, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 1024, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<8, 8, 512, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 512, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<2, 8, 512, 1>, lim));
    for (int W : {4, 8})
        for (int kr : {4, 8})
            for (int n : {256, 512, 1024, 0})
                for (int rot : {0, 1}) {
                    const void* f = W == 8 ? persist_fn_w<8>(kr, n, rot) : persist_fn_w<4>(kr, n, rot);
                    CU(set_smem_attr_one(f, lim));
                }
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 1, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 0, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 1, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 8, 0, 1, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 0, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32<4, 4, 0, 1, 1>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<8, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<4, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<2, 0>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<8, 256>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<4, 256>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<2, 256>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<8, 1024>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<4, 1024>, lim));
    CU(set_smem_attr_one(step_kernel_f32x2<2, 1024>, lim));
    CU(set_smem_attr_one(haissinski_kernel<float>, lim));
    CU(set_smem_attr_one(haissinski_kernel<double>, lim));
    CU(cudaFuncSetAttribute(power_spectrum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(3 * 8192 * sizeof(float2))));
    CU(cudaFuncSetAttribute(spectrogram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(3 * 8192 * sizeof(float2))));
    g_kernels_ready = 1;
    return VFPS_OK;
}

// A group made of one instance, using its own descriptor and tile table.
Group single_group(const Instance& I)
{
    Group g;
    g.prec = I.p.precision;
    g.ni = I.p.interp_points;
    g.var = !I.fast ? 0 : (I.p.clamp ? 2 : (I.p.interp_points != 4 ? 1 : 0));
    g.W = I.W;
    g.fast = I.fast;
    g.kr = fast_kr(I.p.n);
    g.n = I.p.n;
    g.rot = I.p.rotation;
    g.smem = I.fast ? std::max(fast_smem(&I.p, I.W), step_smem(&I.p, I.W)) : step_smem(&I.p, I.W);
    g.ntiles = I.ntiles;
    g.ddescs = I.ddesc;
    g.dtiles = I.dtiles;
    g.dsegs = I.dsegs;
    g.grid = I.ntiles;
    return g;
}

// Recompute the wake, profile and power of the current state of one instance.
int prologue(Instance& I, cudaStream_t s)
{
    int rc = upload_desc(I, s);
    if (rc) return rc;
    Group g = single_group(I);
    return launch_project(g, s);
}

// Haissinski start (vfps_haissinski.cuh): solve for rho_H in one CTA, and if
// it converged write psi = rho_H(q) g(p) as the current state and recompute
// the wake and kick table of that state.  The column-sum and profile buffers
// are the solver's scratch; the moments buffer holds its two result words.
template <typename T>
int haissinski_t(Instance& I, cudaStream_t s, double tol, int max_iter, int32_t* iters)
{
    const size_t sm = vfps::haissinski_smem(I.M, I.n);
    if ((long long)sm > device_smem_limit() - 1024) return VFPS_EINVAL;
    int* info_d = reinterpret_cast<int*>(I.mom);
    haissinski_kernel<T><<<1, 256, sm, s>>>((const Desc<T>*)I.ddesc, I.S, tol, max_iter, I.rho, I.colsum, info_d);
    CU(cudaGetLastError());
    int info[2] = {0, 0};
    CU(cudaMemcpyAsync(info, info_d, sizeof(info), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (iters) *iters = info[0];
    if (!info[1]) {
        // the state is untouched; restore the profile buffers the solver used
        const int rc = prologue(I, s);
        return rc ? rc : VFPS_ECONVERGE;
    }
    DevState st{};
    CU(cudaMemcpyAsync(&st, I.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int nb = (int)std::min<long long>(1024, ((long long)I.n * I.n + 255) / 256);
    outer_state_kernel<T><<<nb, 256, 0, s>>>((const Desc<T>*)I.ddesc, I.rho, I.colsum);
    CU(cudaGetLastError());
    st.scale = 1.0;
    st.ticket = 0;
    CU(cudaMemcpyAsync(I.st, &st, sizeof(DevState), cudaMemcpyHostToDevice, s));
    return prologue(I, s);
}

int instance_haissinski(Instance& I, cudaStream_t s, double tol, int32_t max_iter, int32_t* iters)
{
    if (!(tol > 0.0) || max_iter < 1) return VFPS_EINVAL;
    return I.p.precision ? haissinski_t<double>(I, s, tol, max_iter, iters)
                         : haissinski_t<float>(I, s, tol, max_iter, iters);
}

// Status word -> API code.  -100 - k: the debug build's index check k failed.
int status_code(int status)
{
    if (status <= -100) {
        std::snprintf(g_last_error, sizeof(g_last_error), "debug build: index check %d failed", -100 - status);
        return VFPS_EBOUNDS;
    }
    return status;
}

int read_status(Instance& I, cudaStream_t s)
{
    DevState* st = reinterpret_cast<DevState*>(host_stage().get(kStageHead));
    if (!st) return VFPS_ENOMEM;
    CU(cudaMemcpyAsync(st, I.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return status_code(st->status);
}

// Move the moment records of states t in (mdrained, steps_queued] with t a
// multiple of mom_every to the host (synchronises).  The ring holds the last
// `ring` states, and the callers keep steps_queued - drained below that.
int drain_moments(Instance& I, cudaStream_t s)
{
    const long long lo = I.mdrained + 1, hi = I.steps_queued;
    if (!I.mring || I.mom_every <= 0 || hi < lo) {
        I.mdrained = std::max(I.mdrained, hi);
        return VFPS_OK;
    }
    const long long cnt = hi - lo + 1, mask = I.ring - 1;
    double* hm = reinterpret_cast<double*>(host_stage().get(4 * sizeof(double) * cnt));
    if (!hm) return VFPS_ENOMEM;
    const long long a = lo & mask, first = std::min<long long>(cnt, I.ring - a);
    CU(cudaMemcpyAsync(hm, I.mring + 4 * a, 4 * sizeof(double) * first, cudaMemcpyDeviceToHost, s));
    if (cnt > first)
        CU(cudaMemcpyAsync(hm + 4 * first, I.mring, 4 * sizeof(double) * (cnt - first), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (long long t = lo; t <= hi; ++t) {
        if (t % I.mom_every) continue;
        const double* r = hm + 4 * (t - lo);
        I.mw.insert(I.mw.end(), {(double)t, r[0], r[1], r[2], r[3]});
    }
    I.mdrained = hi;
    return VFPS_OK;
}

int drain(Instance& I, cudaStream_t s);

// Turn the epilogue's moment records on every `every` steps (0: off).  Drains
// what was recorded so far; allocates the ring on first use; the descriptor
// is re-uploaded (callers that copy descriptors must refresh their copies).
int set_moment_recording(Instance& I, cudaStream_t s, int every)
{
    if (every < 0) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(s));
    int rc = drain(I, s);
    if (rc) return rc;
    if (every > 0 && !I.mring) {
        if (dev_alloc((void**)&I.mring, sizeof(double) * 4 * (size_t)I.ring) != cudaSuccess) {
            cudaGetLastError();
            I.mring = nullptr;
            return VFPS_ENOMEM;
        }
    }
    I.mom_every = every;
    I.mdrained = I.steps_queued;
    rc = upload_desc(I, s);
    if (rc) return rc;
    CU(cudaStreamSynchronize(s));
    return VFPS_OK;
}

// Up to cap records (5 doubles each) from the drained moment series.
int64_t take_moments(Instance& I, double* out, int64_t cap, bool consume)
{
    const int64_t have = (int64_t)(I.mw.size() - I.mw_taken) / 5;
    const int64_t k = std::min<int64_t>(cap, have);
    std::memcpy(out, I.mw.data() + I.mw_taken, sizeof(double) * 5 * k);
    if (consume) {
        I.mw_taken += 5 * k;
        if (I.mw_taken == I.mw.size()) {
            I.mw.clear();
            I.mw_taken = 0;
        }
    }
    return k;
}

// Move ring entries [drained, steps_queued) to the host series (synchronises).
int drain(Instance& I, cudaStream_t s)
{
    long long lo = I.drained, hi = I.steps_queued;
    if (hi <= lo) return drain_moments(I, s);
    // only the new entries: [lo, hi) wraps around the ring at most once
    const long long cnt = hi - lo, mask = I.ring - 1;
    double* hp = reinterpret_cast<double*>(host_stage().get(2 * sizeof(double) * cnt));
    if (!hp) return VFPS_ENOMEM;
    double* hq = hp + cnt;
    const long long a = lo & mask, first = std::min<long long>(cnt, I.ring - a);
    CU(cudaMemcpyAsync(hp, I.pring + a, sizeof(double) * first, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(hq, I.qring + a, sizeof(double) * first, cudaMemcpyDeviceToHost, s));
    if (cnt > first) {
        CU(cudaMemcpyAsync(hp + first, I.pring, sizeof(double) * (cnt - first), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(hq + first, I.qring, sizeof(double) * (cnt - first), cudaMemcpyDeviceToHost, s));
    }
    CU(cudaStreamSynchronize(s));
    I.pw.insert(I.pw.end(), hp, hp + cnt);
    I.qw.insert(I.qw.end(), hq, hq + cnt);
    I.drained = hi;
    return drain_moments(I, s);
}

int copy_state(Instance& I, cudaStream_t s, double* psi_out)
{
    const int n = I.n;
    const size_t es = elem_size(&I.p), bytes = (size_t)n * I.ld * es;
    unsigned char* hs = host_stage().get(kStageHead + bytes);
    if (!hs) return VFPS_ENOMEM;
    const DevState& st = *reinterpret_cast<const DevState*>(hs);
    CU(cudaMemcpyAsync(hs, I.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const unsigned char* buf = hs + kStageHead;
    CU(cudaMemcpyAsync(hs + kStageHead, I.psi[st.parity], bytes, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const double scale = st.scale;
    for (int i = 0; i < n; ++i) {
        double* o = psi_out + (size_t)i * n;
        if (es == 8) {
            const double* r = reinterpret_cast<const double*>(buf) + (size_t)i * I.ld;
            for (int j = 0; j < n; ++j) o[j] = r[j] * scale;
        } else {
            const float* r = reinterpret_cast<const float*>(buf) + (size_t)i * I.ld;
            for (int j = 0; j < n; ++j) o[j] = (double)r[j] * scale;
        }
    }
    return status_code(st.status);
}

// Bunch moments of the current state on the device (two small kernels on
// the instance's descriptor and tile table), copied to out[4].  Synchronises.
template <typename T, int W>
int launch_moments_t(Instance& I, cudaStream_t s)
{
    moments_columns_kernel<T, W><<<I.ntiles, W * 32, 0, s>>>((const Desc<T>*)I.ddesc, I.dtiles, I.mom);
    CU(cudaGetLastError());
    moments_finish_kernel<T><<<1, 256, 0, s>>>((const Desc<T>*)I.ddesc, I.mom);
    CU(cudaGetLastError());
    return VFPS_OK;
}

template <typename T>
int launch_moments_p(Instance& I, cudaStream_t s)
{
    switch (I.W) {
    case 8: return launch_moments_t<T, 8>(I, s);
    case 4: return launch_moments_t<T, 4>(I, s);
    case 2: return launch_moments_t<T, 2>(I, s);
    }
    return VFPS_EINVAL;
}

// Power spectrum of the last L CSR-power values of an instance, computed on
// the device, copied to out (L/2 + 1 doubles).  Synchronises.
int instance_power_spectrum(Instance& I, cudaStream_t s, int L, double* out)
{
    if (!out || L < 16 || L > 8192 || (L & (L - 1)) || L > I.ring - 1 || L > I.steps_queued) return VFPS_EINVAL;
    double* d = nullptr;
    CU(cudaMallocAsync((void**)&d, sizeof(double) * (L / 2 + 1), s));
    const size_t sm = (size_t)3 * L * sizeof(float2);
    power_spectrum_kernel<<<1, 256, sm, s>>>(I.pring, I.ring - 1, I.steps_queued - L, L, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * (L / 2 + 1), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) {
        std::snprintf(g_last_error, sizeof(g_last_error), "power spectrum: %s", cudaGetErrorString(e));
        return VFPS_ECUDA;
    }
    return read_status(I, s);
}

// Spectrogram of the CSR-power series of several instances (Sec. IV.C: the
// Fourier transform of P(t) over successive windows): count windows of L
// values, hop steps apart, the last ending at each instance's latest entry,
// one CTA per (window, instance), one launch.  out: nslots x count x (L/2+1)
// doubles.  Synchronises.
int spectrogram(Instance* const* inst, int nslots, int L, int hop, int count, cudaStream_t s, double* out)
{
    if (!out || nslots < 1 || nslots > 65535 || L < 16 || L > 8192 || (L & (L - 1)) || hop < 1 || count < 1)
        return VFPS_EINVAL;
    const long long span = (long long)L + (long long)(count - 1) * hop;
    std::vector<SpecSeries> tab((size_t)nslots);
    for (int i = 0; i < nslots; ++i) {
        const Instance& I = *inst[i];
        if (span > I.ring - 1 || span > I.steps_queued) return VFPS_EINVAL;
        tab[(size_t)i] = SpecSeries{I.pring, (long long)I.ring - 1, I.steps_queued - span};
    }
    const size_t rows = (size_t)nslots * count, outb = rows * (size_t)(L / 2 + 1) * sizeof(double);
    const size_t tab_off = align_up(outb, kAlign), total = tab_off + sizeof(SpecSeries) * tab.size();
    unsigned char* d = nullptr;
    CU(cudaMallocAsync((void**)&d, total, s));
    cudaError_t e = cudaMemcpyAsync(d + tab_off, tab.data(), sizeof(SpecSeries) * tab.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        spectrogram_kernel<<<dim3((unsigned)count, (unsigned)nslots), 256, (size_t)3 * L * sizeof(float2), s>>>(
            (const SpecSeries*)(d + tab_off), L, hop, (double*)d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, outb, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        note_cuda_error(e, "spectrogram");
        return VFPS_ECUDA;
    }
    for (int i = 0; i < nslots; ++i) {
        const int rc = read_status(*inst[i], s);
        if (rc) return rc;
    }
    return VFPS_OK;
}

int instance_moments(Instance& I, cudaStream_t s, double* out)
{
    if (!out) return VFPS_EINVAL;
    int rc = I.p.precision ? launch_moments_p<double>(I, s) : launch_moments_p<float>(I, s);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, I.mom + 3 * I.n, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    return read_status(I, s);
}

}  // namespace

// ============================================================================
// Single-simulation handle
struct vfps_handle {
    Instance* I = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    int persist = -1;  // persistent launches: -1 not decided yet, 0 off, 1 on
};

extern "C" {

void vfps_params_default(vfps_params* p)
{
    if (!p) return;
    p->n = 256;
    p->steps_per_period = 1000;
    p->interp_points = 4;
    p->clamp = 0;
    p->fp_derivative = 1;
    p->pad_factor = 2;
    p->precision = 0;
    p->renormalize = 1;
    p->rotation = 0;
    p->half_width = 6.0;
    p->beta = 0.0;
}

const char* vfps_last_cuda_error(void) { return g_last_error; }

const char* vfps_strerror(int code)
{
    switch (code) {
    case VFPS_OK: return "ok";
    case VFPS_EINVAL: return "invalid argument";
    case VFPS_ENOMEM: return "out of memory";
    case VFPS_ECUDA: return "CUDA runtime error";
    case VFPS_ETIMEOUT: return "bounded device wait timed out";
    case VFPS_ENAN: return "non-finite or non-positive charge";
    case VFPS_EBUSY: return "capacity exhausted";
    case VFPS_EBOUNDS: return "index check failed (debug build)";
    case VFPS_ECONVERGE: return "iteration did not converge";
    }
    return "unknown error";
}

int vfps_create(const vfps_params* params, const double* psi0, void* cuda_stream, vfps_handle** out)
{
    if (!out) return VFPS_EINVAL;
    *out = nullptr;
    std::unique_ptr<vfps_handle> h(new (std::nothrow) vfps_handle());
    if (!h) return VFPS_ENOMEM;
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    Instance* I = nullptr;
    int rc = init_kernels();
    if (rc == VFPS_OK) rc = create_instance(params, psi0, kRingDefault, h->stream, &I, true);
    if (rc) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        return rc;
    }
    h->I = I;
    // lone FP32 simulations step in persistent launches unless
    // VFPS_PERSISTENT=0; the bounded waits of those launches give up after
    // VFPS_SPIN_LIMIT polls, and VFPS_FAULT_NO_SIGNAL=1 (tests) makes the
    // finaliser CTA withhold its kick tables so that they do
    if (const char* e = std::getenv("VFPS_PERSISTENT")) h->persist = (e[0] == '0') ? 0 : -1;
    if (const char* e = std::getenv("VFPS_SPIN_LIMIT")) {
        const long long v = std::atoll(e);
        if (v > 0 && v < (1LL << 31)) I->spin_limit = (unsigned)v;
    }
    if (const char* e = std::getenv("VFPS_FAULT_NO_SIGNAL")) I->fault_no_signal = (e[0] == '1');
    rc = upload_desc(*I, h->stream);
    if (rc == VFPS_OK) rc = prologue(*I, h->stream);
    if (rc) {
        destroy_instance(I);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        return rc;
    }
    *out = h.release();
    return VFPS_OK;
}

int vfps_set_impedance(vfps_handle* h, int model, double Pi, double S_csr, const double* table)
{
    if (!h) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    int rc = upload_impedance(*h->I, model, Pi, S_csr, table, h->stream);
    if (rc) return rc;
    return prologue(*h->I, h->stream);
}

static int ensure_graph(vfps_handle* h)
{
    if (h->graph) return VFPS_OK;
    Group g = single_group(*h->I);
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = VFPS_OK;
    for (int i = 0; i < kGraphSteps && rc == VFPS_OK; ++i) rc = launch_step(g, h->stream);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (rc) return rc;
    if (e != cudaSuccess) return VFPS_ECUDA;
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return VFPS_ECUDA;
    }
    return VFPS_OK;
}

// Persistent launches apply when the simulation's kernel has a persistent
// form and all its CTAs plus the finaliser fit on the device at once.
static bool use_persistent(vfps_handle* h, const Group& g)
{
    if (h->persist < 0) {
        h->persist = 0;
        const void* f = persist_fn(g);
        int per_sm = 0;
        if (f && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, group_threads(g), g.smem) ==
                     cudaSuccess &&
            (long long)per_sm * num_sms() >= (long long)g.grid + 1)
            h->persist = 1;
    }
    return h->persist == 1;
}

int vfps_step(vfps_handle* h, int64_t nsteps)
{
    if (!h || nsteps < 0) return VFPS_EINVAL;
    Range r("vfps_step");
    Instance& I = *h->I;
    Group g = single_group(I);
    const bool persist = use_persistent(h, g);
    int rc;
    while (nsteps > 0) {
        // keep the ring from overwriting undrained entries
        long long room = (long long)I.ring - 1 - (I.steps_queued - I.drained);
        if (room <= 0) {
            rc = drain(I, h->stream);
            if (rc) return rc;
            continue;
        }
        long long chunk = std::min<long long>(nsteps, room);
        if (persist) {
            chunk = std::min<long long>(chunk, kPersistSteps);
            rc = launch_persistent(g, I, (int)chunk, h->stream);
            if (rc) return rc;
        } else if (chunk >= kGraphSteps) {
            rc = ensure_graph(h);
            if (rc) return rc;
            long long ng = chunk / kGraphSteps;
            for (long long i = 0; i < ng; ++i) CU(cudaGraphLaunch(h->graph, h->stream));
            chunk = ng * kGraphSteps;
        } else {
            for (long long i = 0; i < chunk; ++i) {
                rc = launch_step(g, h->stream);
                if (rc) return rc;
            }
        }
        I.steps_queued += chunk;
        nsteps -= chunk;
    }
    return VFPS_OK;
}

int vfps_power_spectrum(vfps_handle* h, int32_t length, double* out)
{
    if (!h) return VFPS_EINVAL;
    return instance_power_spectrum(*h->I, h->stream, length, out);
}

int vfps_moments(vfps_handle* h, double* out)
{
    if (!h) return VFPS_EINVAL;
    return instance_moments(*h->I, h->stream, out);
}

int vfps_record_moments(vfps_handle* h, int32_t every)
{
    if (!h || every < 0) return VFPS_EINVAL;
    return set_moment_recording(*h->I, h->stream, every);
}

int vfps_moment_series(vfps_handle* h, double* out, int64_t cap, int64_t* n_written)
{
    if (!h || !n_written || cap < 0 || (cap > 0 && !out)) return VFPS_EINVAL;
    Instance& I = *h->I;
    int rc = drain(I, h->stream);
    if (rc) return rc;
    *n_written = take_moments(I, out, cap, true);
    return read_status(I, h->stream);
}

int vfps_spectrogram(vfps_handle* h, int32_t length, int32_t hop, int32_t count, double* out)
{
    if (!h) return VFPS_EINVAL;
    Instance* I = h->I;
    return spectrogram(&I, 1, length, hop, count, h->stream, out);
}

int vfps_profile(vfps_handle* h, double* rho_out)
{
    if (!h || !rho_out) return VFPS_EINVAL;
    CU(cudaMemcpyAsync(rho_out, h->I->rho, sizeof(double) * h->I->n, cudaMemcpyDeviceToHost, h->stream));
    return read_status(*h->I, h->stream);
}

static int drain_series(vfps_handle* h, bool power, double* out, int64_t cap, int64_t* n_written)
{
    if (!h || !n_written || cap < 0 || (cap > 0 && !out)) return VFPS_EINVAL;
    Instance& I = *h->I;
    int rc = drain(I, h->stream);
    if (rc) return rc;
    std::vector<double>& v = power ? I.pw : I.qw;
    size_t& taken = power ? I.pw_taken : I.qw_taken;
    int64_t k = std::min<int64_t>(cap, (int64_t)(v.size() - taken));
    for (int64_t i = 0; i < k; ++i) out[i] = v[taken + i];
    taken += k;
    *n_written = k;
    if (I.pw_taken == I.pw.size() && I.qw_taken == I.qw.size()) {
        I.pw.clear();
        I.qw.clear();
        I.pw_taken = I.qw_taken = 0;
    }
    return read_status(I, h->stream);
}

int vfps_csr_power(vfps_handle* h, double* out, int64_t cap, int64_t* n_written)
{
    return drain_series(h, true, out, cap, n_written);
}

int vfps_charge_series(vfps_handle* h, double* out, int64_t cap, int64_t* n_written)
{
    return drain_series(h, false, out, cap, n_written);
}

int vfps_get_state(vfps_handle* h, double* psi_out)
{
    if (!h || !psi_out) return VFPS_EINVAL;
    return copy_state(*h->I, h->stream, psi_out);
}

int vfps_set_state(vfps_handle* h, const double* psi)
{
    if (!h || !psi) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    int rc = upload_psi(*h->I, psi, h->stream);
    if (rc) return rc;
    return prologue(*h->I, h->stream);
}

// Checkpoint: the state exactly as the device holds it between steps.
struct vfps_checkpoint_head {
    char magic[8];          // "VFPSCKP1"
    vfps_params params;     // must match the loading handle's
    int32_t model, pad0;
    double Pi, S;           // impedance of the run (must match)
    int32_t n, ld, M, es;
    DevState st;            // pending scale, step count, parity (ticket 0)
    double p_t, q_t;        // ring entries of step t: P(psi_t), charge of the step that made psi_t
};

static size_t checkpoint_bytes(const Instance& I)
{
    const size_t es = elem_size(&I.p);
    return sizeof(vfps_checkpoint_head) + (size_t)I.n * I.ld * es + (size_t)I.n * es + (size_t)I.n * 32 +
           (size_t)I.n * 8;
}

int vfps_checkpoint_bytes(vfps_handle* h, int64_t* bytes)
{
    if (!h || !bytes) return VFPS_EINVAL;
    *bytes = (int64_t)checkpoint_bytes(*h->I);
    return VFPS_OK;
}

int vfps_save_checkpoint(vfps_handle* h, void* buf, int64_t bytes)
{
    if (!h || !buf || bytes < (int64_t)checkpoint_bytes(*h->I)) return VFPS_EINVAL;
    Instance& I = *h->I;
    const size_t es = elem_size(&I.p);
    unsigned char* o = (unsigned char*)buf;
    vfps_checkpoint_head hd{};
    std::memcpy(hd.magic, "VFPSCKP1", 8);
    hd.params = I.p;
    hd.model = I.model;
    hd.Pi = I.Pi;
    hd.S = I.S;
    hd.n = I.n;
    hd.ld = I.ld;
    hd.M = I.M;
    hd.es = (int32_t)es;
    CU(cudaMemcpyAsync(&hd.st, I.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    const long long t = hd.st.t, mask = I.ring - 1;
    CU(cudaMemcpyAsync(&hd.p_t, I.pring + (t & mask), sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&hd.q_t, I.qring + ((t - 1) & mask), sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    size_t off = sizeof(hd);
    CU(cudaMemcpyAsync(o + off, I.psi[hd.st.parity], (size_t)I.n * I.ld * es, cudaMemcpyDeviceToHost, h->stream));
    off += (size_t)I.n * I.ld * es;
    CU(cudaMemcpyAsync(o + off, I.kick, (size_t)I.n * es, cudaMemcpyDeviceToHost, h->stream));
    off += (size_t)I.n * es;
    CU(cudaMemcpyAsync(o + off, I.kickw, (size_t)I.n * 32, cudaMemcpyDeviceToHost, h->stream));
    off += (size_t)I.n * 32;
    CU(cudaMemcpyAsync(o + off, I.rho, (size_t)I.n * 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    hd.st.ticket = 0;
    std::memcpy(o, &hd, sizeof(hd));
    return status_code(hd.st.status);
}

int vfps_load_checkpoint(vfps_handle* h, const void* buf, int64_t bytes)
{
    if (!h || !buf || bytes < (int64_t)sizeof(vfps_checkpoint_head)) return VFPS_EINVAL;
    Instance& I = *h->I;
    vfps_checkpoint_head hd;
    std::memcpy(&hd, buf, sizeof(hd));
    const size_t es = elem_size(&I.p);
    const vfps_params &a = hd.params, &q = I.p;  // field by field: the struct has padding bytes
    const bool same = a.n == q.n && a.steps_per_period == q.steps_per_period && a.interp_points == q.interp_points &&
                      a.clamp == q.clamp && a.fp_derivative == q.fp_derivative && a.pad_factor == q.pad_factor &&
                      a.precision == q.precision && a.renormalize == q.renormalize && a.rotation == q.rotation &&
                      a.half_width == q.half_width && a.beta == q.beta;
    if (std::memcmp(hd.magic, "VFPSCKP1", 8) || !same ||
        hd.model != I.model || hd.Pi != I.Pi || hd.S != I.S || hd.n != I.n || hd.ld != I.ld || hd.M != I.M ||
        hd.es != (int32_t)es || bytes < (int64_t)checkpoint_bytes(I) || hd.st.parity < 0 || hd.st.parity > 1 ||
        hd.st.t < 0)
        return VFPS_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    const unsigned char* in = (const unsigned char*)buf;
    size_t off = sizeof(hd);
    CU(cudaMemcpyAsync(I.psi[hd.st.parity], in + off, (size_t)I.n * I.ld * es, cudaMemcpyHostToDevice, h->stream));
    off += (size_t)I.n * I.ld * es;
    CU(cudaMemcpyAsync(I.kick, in + off, (size_t)I.n * es, cudaMemcpyHostToDevice, h->stream));
    off += (size_t)I.n * es;
    CU(cudaMemcpyAsync(I.kickw, in + off, (size_t)I.n * 32, cudaMemcpyHostToDevice, h->stream));
    off += (size_t)I.n * 32;
    CU(cudaMemcpyAsync(I.rho, in + off, (size_t)I.n * 8, cudaMemcpyHostToDevice, h->stream));
    const long long t = hd.st.t, mask = I.ring - 1;
    CU(cudaMemcpyAsync(I.pring + (t & mask), &hd.p_t, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(I.qring + ((t - 1) & mask), &hd.q_t, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DevState st = hd.st;
    st.ticket = 0;
    CU(cudaMemcpyAsync(I.st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    // the host bookkeeping restarts at step t: series drained from there on
    I.steps_queued = I.drained = I.mdrained = t;
    I.pw.clear();
    I.qw.clear();
    I.mw.clear();
    I.pw_taken = I.qw_taken = I.mw_taken = 0;
    return status_code(st.status);
}

int vfps_haissinski(vfps_handle* h, double tol, int32_t max_iter, int32_t* iterations)
{
    if (!h) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    return instance_haissinski(*h->I, h->stream, tol, max_iter, iterations);
}

int vfps_steps_done(vfps_handle* h, int64_t* steps)
{
    if (!h || !steps) return VFPS_EINVAL;
    *steps = h->I->steps_queued;
    return VFPS_OK;
}

int vfps_step_mode(vfps_handle* h, int32_t* persistent)
{
    if (!h || !persistent) return VFPS_EINVAL;
    *persistent = use_persistent(h, single_group(*h->I)) ? 1 : 0;
    return VFPS_OK;
}

int vfps_destroy(vfps_handle* h)
{
    if (!h) return VFPS_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    destroy_instance(h->I);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return VFPS_OK;
}

// Host-only helper (no device needed): the library's own impedance table for
// a grid, as interleaved (re, im) pairs, M/2+1 of them.
int vfps_impedance_table(int model, int32_t n, double half_width, int32_t pad_factor, double Pi,
                         double* out_re_im)
{
    if (!out_re_im || n < 8 || n > 2048 || pad_factor < 2 || pad_factor > 64 || !(half_width > 0.0))
        return VFPS_EINVAL;
    if ((long long)pad_factor * n > 16384) return VFPS_EINVAL;
    if (model < 0 || model > 2 || (model == 2 && !(Pi > 0.0))) return VFPS_EINVAL;
    vfps_params tmp{};
    tmp.n = n;
    tmp.pad_factor = pad_factor;
    int M = fft_length(&tmp);
    std::vector<std::complex<double>> z;
    vfps::impedance_table(model, M, 2.0 * half_width / (n - 1), Pi, z);
    for (size_t k = 0; k < z.size(); ++k) {
        out_re_im[2 * k] = z[k].real();
        out_re_im[2 * k + 1] = z[k].imag();
    }
    return VFPS_OK;
}

}  // extern "C"

// ============================================================================
// Batch of slots (vfps_batch_*)
struct vfps_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int max_slots = 0;
    long long budget = 0;
    long long used = 0;
    std::vector<Instance*> slots;  // nullptr = free
    std::vector<Group> groups;
    bool dirty = true;             // active set changed: rebuild groups
    void* gmem = nullptr;          // descriptor and tile arrays of the groups
    size_t gbytes = 0;
    std::vector<cudaStream_t> pool;   // one stream per group, forked from `stream`
    std::vector<cudaEvent_t> events;  // fork event + one join event per pool stream
    std::vector<cudaEvent_t> timers;  // two timing events per pool stream (autotuner)
    std::vector<unsigned char> hbuf;  // host copy of gmem
    bool autotune = true;
    bool pairing = false;             // vfps_batch_pairing: pair kernel for equal geometries
    int pin_W = 0, pin_tps = 0;       // vfps_batch_pin_shape: fixed shape of FP32 groups
    // kGraphSteps steps of the current group layout (fork, every group's
    // launches on its stream, join) captured as one CUDA graph; dropped
    // whenever a layout changes
    cudaGraphExec_t graph = nullptr;
    // admissions set up new slots (upload, prologue) on their own stream, so
    // that a vfps_batch_add never waits for the chunk in flight; the batch
    // stream waits for that set-up before its next work
    cudaStream_t adm = nullptr;
    cudaEvent_t adm_ev = nullptr;
};

namespace {

long long remaining(const Instance* I) { return I->target - I->steps_queued; }

void drop_graph(vfps_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

void free_groups(vfps_batch* b)
{
    drop_graph(b);
    if (b->gmem) cudaFree(b->gmem);
    b->gmem = nullptr;
    b->gbytes = 0;
    b->groups.clear();
}

// CTAs of an FP32 group's kernel that fit on one SM at width W with smem
// bytes of dynamic shared memory.
template <typename K>
int blocks_per_sm(K kernel, int threads, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(nb, 1);
}

template <int W>
int fast_blocks_t(const Group& g, size_t smem)
{
    if (g.var == 2) {
        if (g.kr == 8)
            return blocks_per_sm(g.rot ? step_kernel_f32<4, 8, 0, 1, 1> : step_kernel_f32<4, 8, 0, 0, 1>, 128, smem);
        return blocks_per_sm(g.rot ? step_kernel_f32<4, 4, 0, 1, 1> : step_kernel_f32<4, 4, 0, 0, 1>, 128, smem);
    }
    if (g.var) {
        if (g.kr == 8)
            return blocks_per_sm(g.rot ? step_kernel_f32<4, 8, 0, 1, 0> : step_kernel_f32<4, 8, 0, 0, 0>, 128, smem);
        return blocks_per_sm(g.rot ? step_kernel_f32<4, 4, 0, 1, 0> : step_kernel_f32<4, 4, 0, 0, 0>, 128, smem);
    }
    if (g.pair) {
        if (g.n == 256) return blocks_per_sm(step_kernel_f32x2<W, 256>, W * 32, smem);
        if (g.n == 1024) return blocks_per_sm(step_kernel_f32x2<W, 1024>, W * 32, smem);
        return blocks_per_sm(step_kernel_f32x2<W, 0>, W * 32, smem);
    }
    if (g.kr == 8) {
        if (g.n == 256)
            return blocks_per_sm(g.rot ? step_kernel_f32<W, 8, 256, 1> : step_kernel_f32<W, 8, 256, 0>, W * 32, smem);
        if (g.n == 1024)
            return blocks_per_sm(g.rot ? step_kernel_f32<W, 8, 1024, 1> : step_kernel_f32<W, 8, 1024, 0>,
                                 fast_threads(W, 1024), smem);
        if (g.n == 512)
            return blocks_per_sm(g.rot ? step_kernel_f32<W, 8, 512, 1> : step_kernel_f32<W, 8, 512, 0>,
                                 fast_threads(W, 512), smem);
        return blocks_per_sm(g.rot ? step_kernel_f32<W, 8, 0, 1> : step_kernel_f32<W, 8, 0, 0>, W * 32, smem);
    }
    return blocks_per_sm(g.rot ? step_kernel_f32<W, 4, 0, 1> : step_kernel_f32<W, 4, 0, 0>, W * 32, smem);
}

int fast_blocks(const Group& g, int W, size_t smem)
{
    switch (W) {
    case 8: return fast_blocks_t<8>(g, smem);
    case 4: return fast_blocks_t<4>(g, smem);
    default: return fast_blocks_t<2>(g, smem);
    }
}

// Shared memory of a group member's kernel at CTA width W.
size_t member_smem(const Group& g, const Instance* I, int W)
{
    return g.pair ? pair_smem(&I->p, W) : fast_smem(&I->p, W);
}

// Tiles (CTA column blocks) of one step of a group at width W: a pair
// group's tiles cover both simulations of a pair.
int group_tiles(const Group& g, int W)
{
    int nt = 0;
    for (const Instance* I : g.members) nt += (I->n + W - 1) / W;
    return g.pair ? nt / 2 : nt;
}

// Lay out a batch group for CTA width W in the host copy of the group
// arrays: its members' descriptors (ntiles patched to the CTAs that touch
// each simulation per step) and its tile table.  FP32 groups get segments
// (unit, first column, tiles): strips of tps tiles, one per CTA, or with
// tps = -1 a balanced grid of one resident wave's share of CTAs, each taking
// an equal run of the group's tiles split at simulation boundaries.  Other
// groups get one tile per CTA.  Returns false if the segments do not fit.
bool layout_group(vfps_batch* b, Group& g, int W, int tps)
{
    const size_t dsz = g.prec ? sizeof(Desc<double>) : sizeof(Desc<float>);
    size_t smem = 0;
    for (const Instance* I : g.members) {
        smem = std::max(smem, step_smem(&I->p, W));
        if (g.fast) smem = std::max(smem, member_smem(g, I, W));
    }
    if (!g.fast) {
        int2* ht = (int2*)(b->hbuf.data() + g.off_t);
        int nt = 0;
        for (size_t k = 0; k < g.members.size(); ++k) {
            Instance* I = g.members[k];
            unsigned char* hd = b->hbuf.data() + g.off_d + k * dsz;
            std::memcpy(hd, I->hdesc, dsz);
            const int per_inst = (I->n + W - 1) / W;
            for (int t = 0; t < per_inst; ++t) ht[nt++] = make_int2((int)k, t * W);
            if (g.prec) ((Desc<double>*)hd)->ntiles = per_inst;
            else ((Desc<float>*)hd)->ntiles = per_inst;
        }
        g.W = W;
        g.tps = 1;
        g.smem = smem;
        g.ntiles = nt;
        g.tab_bytes = g.off_t + sizeof(int2) * nt - g.off_d;
        return true;
    }
    const int units = g.pair ? (int)g.members.size() / 2 : (int)g.members.size();
    const int per = (g.n + W - 1) / W;  // tiles per unit (a group shares n)
    std::vector<int4> segs;
    std::vector<int> touch(units, 0);
    int spc = 1, grid = 0;
    if (tps > 0) {
        for (int u = 0; u < units; ++u)
            for (int k = 0; k < per / tps; ++k) segs.push_back(make_int4(u, k * tps * W, tps, 0));
        std::fill(touch.begin(), touch.end(), per / tps);
        grid = (int)segs.size();
    } else {
        const long long NT = (long long)units * per;
        const int nb = fast_blocks(g, W, smem);
        long long G = std::llround(g.share * nb * num_sms());
        G = std::max(1LL, std::min(G, NT));
        std::vector<std::vector<int4>> cta((size_t)G);
        for (long long c = 0; c < G; ++c) {
            long long t = c * NT / G;
            const long long t1 = (c + 1) * NT / G;
            while (t < t1) {
                const int u = (int)(t / per), loc = (int)(t % per);
                const int len = (int)(std::min(t1, (long long)(u + 1) * per) - t);
                cta[(size_t)c].push_back(make_int4(u, loc * W, len, 0));
                ++touch[u];
                t += len;
            }
            spc = std::max(spc, (int)cta[(size_t)c].size());
        }
        for (auto& v : cta) {
            v.resize((size_t)spc, make_int4(0, 0, 0, 0));
            segs.insert(segs.end(), v.begin(), v.end());
        }
        grid = (int)G;
    }
    if (segs.size() > g.seg_cap) return false;
    for (size_t k = 0; k < g.members.size(); ++k) {
        unsigned char* hd = b->hbuf.data() + g.off_d + k * dsz;
        std::memcpy(hd, g.members[k]->hdesc, dsz);
        ((Desc<float>*)hd)->ntiles = touch[g.pair ? k / 2 : k];
    }
    std::memcpy(b->hbuf.data() + g.off_t, segs.data(), sizeof(int4) * segs.size());
    g.W = W;
    g.tps = tps;
    g.smem = smem;
    g.spc = spc;
    g.grid = grid;
    g.ntiles = units * per;
    g.tab_bytes = g.off_t + sizeof(int4) * segs.size() - g.off_d;
    return true;
}

int default_tps(const Group& g, int W)
{
    const int per_inst = (g.n + W - 1) / W;
    const int nt = group_tiles(g, W);
    const int target = 2 * num_sms();
    for (int t = per_inst; t >= 1; --t)
        if (per_inst % t == 0 && (t == 1 || nt / t >= target)) return t;
    return 1;
}

// ---- autotuner: per (n, precision, rotation, steps/period, group size
// rounded up to a power of two, default width) the fastest (W, tps) of the
// FP32 streaming kernel, timed on the group's own first steps.  Every
// candidate computes the same bits (results do not depend on the CTA width or
// the strip length), so the timed steps are ordinary steps of the run.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> g_tuned;
constexpr int kTuneSteps = 16;  // steps timed per candidate (4 were too few to rank 8- and 16-tile strips)

bool autotune_enabled()
{
    const char* e = std::getenv("VFPS_AUTOTUNE");
    return !(e && e[0] == '0');
}

bool tuned_choice(const std::tuple<int, int, int, int, int, int>& key, std::pair<int, int>* out)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
}

// A pinned shape applies to a group if its shared memory fits and the strip
// length divides the tiles per instance.
bool pin_fits(const Group& g, int W, int tps)
{
    const long long lim = device_smem_limit() - 1024;
    if (g.var && W != 4) return false;
    for (const Instance* I : g.members)
        if ((long long)member_smem(g, I, W) > lim) return false;
    return tps == -1 || (tps >= 1 && ((g.n + W - 1) / W) % tps == 0);
}

std::vector<std::pair<int, int>> tune_candidates(const Group& g)
{
    std::vector<std::pair<int, int>> c;
    const long long lim = device_smem_limit() - 1024;
    for (int W : {8, 4, 2}) {
        if (g.var && W != 4) continue;
        bool fits = true;
        for (const Instance* I : g.members) fits = fits && (long long)member_smem(g, I, W) <= lim;
        if (!fits) continue;
        const int per_inst = (g.n + W - 1) / W;
        const int nt = group_tiles(g, W);
        for (int t : {1, 2, 4, 8, 16, 32})
            if (per_inst % t == 0 && nt / t >= num_sms()) c.push_back({W, t});
        if (c.empty() || c.back().first != W) c.push_back({W, default_tps(g, W)});
        c.push_back({W, -1});  // balanced grid
    }
    return c;
}

// Whether two FP32 simulations advance by the same rotation map and
// Fokker-Planck weights (grid, halo, angle, damping): they may then share the
// pair kernel.
bool same_geometry(const Instance& a, const Instance& b)
{
    const Desc<float>& x = *reinterpret_cast<const Desc<float>*>(a.hdesc);
    const Desc<float>& y = *reinterpret_cast<const Desc<float>*>(b.hdesc);
    return x.n == y.n && x.ld == y.ld && x.h == y.h && x.rotation == y.rotation &&
           std::memcmp(&x.cm1, &y.cm1, sizeof(float)) == 0 && std::memcmp(&x.sn, &y.sn, sizeof(float)) == 0 &&
           std::memcmp(&x.c, &y.c, sizeof(float)) == 0 && std::memcmp(x.ga, y.ga, sizeof(x.ga)) == 0 &&
           std::memcmp(x.gb, y.gb, sizeof(x.gb)) == 0;
}

// One launch group to be: its members and kind.
struct GroupPlan {
    std::tuple<int, int, int, int> key;  // precision, (N_I, fast, rotation), W, n
    int pair = 0;
    std::vector<Instance*> members;
};

// Group the slots that still have steps to run by (precision, N_I, W, n):
// one launch per group and step, each group on its own stream so that the
// groups -- and the two halves of a large group -- overlap, and one group's
// tail (its last CTAs and their finalisers) hides behind another's work.
// Grouping by n keeps small grids from running at the occupancy that the
// largest grid's shared memory would impose.  Simulations of equal geometry
// that the pair kernel covers go, two by two, into pair groups; an odd one
// out joins the single-simulation group of its key.
int rebuild_groups(vfps_batch* b)
{
    CU(cudaStreamSynchronize(b->stream));
    free_groups(b);
    std::map<std::tuple<int, int, int, int>, std::vector<Instance*>> by_key;
    for (Instance* I : b->slots)
        if (I && remaining(I) > 0)
            by_key[{I->p.precision, ((I->p.interp_points * 2 + I->p.clamp) * 2 + I->fast) * 2 + I->p.rotation, I->W,
                    I->n}].push_back(I);
    std::vector<GroupPlan> cls;
    auto add_halves = [&](const std::tuple<int, int, int, int>& key, int pair, const std::vector<Instance*>& m) {
        // large groups in two halves (a pair group splits between pairs)
        const size_t unit = pair ? 2 : 1, units = m.size() / unit;
        const size_t cut = units >= 8 / unit ? unit * ((units + 1) / 2) : m.size();
        GroupPlan a{key, pair, std::vector<Instance*>(m.begin(), m.begin() + cut)};
        cls.push_back(a);
        if (cut < m.size()) cls.push_back(GroupPlan{key, pair, std::vector<Instance*>(m.begin() + cut, m.end())});
    };
    for (auto& kv : by_key) {
        std::vector<Instance*> single;
        std::vector<std::vector<Instance*>> sigs;
        for (Instance* I : kv.second) {
            if (!(b->pairing && I->fast && I->mom_every == 0 && pair_eligible(&I->p) &&
                  (long long)pair_smem(&I->p, 2) <= device_smem_limit() - 1024)) {
                single.push_back(I);
                continue;
            }
            bool placed = false;
            for (auto& sg : sigs)
                if (same_geometry(*sg[0], *I)) {
                    sg.push_back(I);
                    placed = true;
                    break;
                }
            if (!placed) sigs.push_back({I});
        }
        for (auto& sg : sigs) {
            if (sg.size() % 2) {
                single.push_back(sg.back());
                sg.pop_back();
            }
            if (!sg.empty()) add_halves(kv.first, 1, sg);
        }
        if (!single.empty()) add_halves(kv.first, 0, single);
    }
    if (cls.empty()) {
        b->dirty = false;
        return VFPS_OK;
    }
    while (b->pool.size() < cls.size()) {
        cudaStream_t st;
        cudaEvent_t ev;
        CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->pool.push_back(st);
        CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->events.push_back(ev);
    }
    if (b->events.size() < b->pool.size() + 1) {
        cudaEvent_t ev;
        CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->events.push_back(ev);
    }
    while (b->timers.size() < 2 * b->pool.size()) {
        cudaEvent_t ev;
        CU(cudaEventCreate(&ev));
        b->timers.push_back(ev);
    }
    // descriptor and tile arrays, with room for the narrowest width (W = 2)
    size_t total = 0;
    std::vector<std::pair<size_t, size_t>> offs;
    // tile or segment tables: room for one strip per tile at W = 2, or a
    // balanced grid of up to 32 CTAs per SM with up to 4 segments each
    std::vector<size_t> caps;
    double fast_cells = 0.0;
    for (auto& kv : cls) {
        size_t nt = 0;
        for (Instance* I : kv.members) {
            nt += (size_t)(I->n + 1) / 2;
            if (I->fast) fast_cells += double(I->n) * I->n;
        }
        const size_t cap = nt + 128 * (size_t)num_sms();
        size_t od = align_up(total, kAlign);
        size_t ot = align_up(od + kv.members.size() * sizeof(Desc<double>), kAlign);
        total = ot + cap * sizeof(int4);
        offs.push_back({od, ot});
        caps.push_back(cap);
    }
    if (dev_alloc(&b->gmem, total) != cudaSuccess) {
        cudaGetLastError();
        return VFPS_ENOMEM;
    }
    b->gbytes = total;
    b->hbuf.assign(total, 0);
    size_t gi = 0;
    for (auto& kv : cls) {
        Group g;
        g.prec = std::get<0>(kv.key);
        g.ni = std::get<1>(kv.key) / 8;
        g.fast = (std::get<1>(kv.key) >> 1) & 1;
        g.var = !g.fast ? 0 : (((std::get<1>(kv.key) >> 2) & 1) ? 2 : (g.ni != 4 ? 1 : 0));
        g.pair = kv.pair;
        g.stream = b->pool[gi];
        g.t0 = b->timers[2 * gi];
        g.t1 = b->timers[2 * gi + 1];
        g.members = kv.members;
        g.off_d = offs[gi].first;
        g.off_t = offs[gi].second;
        g.ddescs = (unsigned char*)b->gmem + g.off_d;
        g.dtiles = (int2*)((unsigned char*)b->gmem + g.off_t);
        g.dsegs = (int4*)((unsigned char*)b->gmem + g.off_t);
        g.seg_cap = caps[gi];
        if (g.fast && fast_cells > 0.0) {
            double cells = 0.0;
            for (const Instance* I : kv.members) cells += double(I->n) * I->n;
            g.share = cells / fast_cells;
        }
        g.kr = fast_kr(kv.members[0]->p.n);  // a group shares n
        g.n = kv.members[0]->p.n;
        g.rot = kv.members[0]->p.rotation;
        int W = std::get<2>(kv.key), tps = 1;
        if (g.pair) {
            // the widest width whose pair-kernel shared memory fits
            const long long lim = device_smem_limit() - 1024;
            for (int w : {8, 4, 2}) {
                bool fits = true;
                for (const Instance* I : g.members) fits = fits && (long long)pair_smem(&I->p, w) <= lim;
                if (fits) {
                    W = w;
                    break;
                }
            }
        }
        if (g.fast) {
            // a strip of tps consecutive tiles per CTA: the largest divisor of
            // the tiles per instance that still leaves two CTAs per SM (long
            // strips spread the CTA prologue and the halo columns over more
            // cells; measured on 512 x N=256: 4 tiles 161 us, 8 152, 16 148);
            // the autotuner replaces this choice once it has timed the group
            tps = default_tps(g, W);
            const Instance* I0 = kv.members[0];
            const int cnt = (int)kv.members.size();
            int bucket = 1;
            while (bucket < cnt) bucket <<= 1;
            g.tune_key = std::make_tuple(I0->n, g.prec, g.rot + 2 * g.pair + 4 * g.ni + 32 * g.var,
                                         I0->p.steps_per_period,
                                         bucket, I0->W);
            std::pair<int, int> best;
            if (b->pin_W && pin_fits(g, b->pin_W, b->pin_tps)) {
                W = b->pin_W;
                tps = b->pin_tps;
            } else if (tuned_choice(g.tune_key, &best)) {
                W = best.first;
                tps = best.second;
            } else if (b->autotune && autotune_enabled()) {
                g.cands = tune_candidates(g);
                g.cand = -1;
            }
        }
        if (!layout_group(b, g, W, tps)) {
            g.cands.clear();
            layout_group(b, g, W, default_tps(g, W));
        }
        b->groups.push_back(g);
        ++gi;
    }
    CU(cudaMemcpyAsync(b->gmem, b->hbuf.data(), total, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    b->dirty = false;
    return VFPS_OK;
}

// After a tuning step: record each tuning group's time, move on to its next
// candidate, and once all are timed keep the fastest (cached per key).
int tune_step_done(vfps_batch* b)
{
    CU(cudaStreamSynchronize(b->stream));
    for (Group& g : b->groups) {
        if (g.cands.empty()) continue;
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, g.t0, g.t1));
        if (g.cand >= 0) g.cand_ms.push_back(ms);  // the warm-up steps (-1) are not kept
        if (++g.cand < (int)g.cands.size()) continue;
        size_t best = 0;
        for (size_t i = 1; i < g.cand_ms.size(); ++i)
            if (g.cand_ms[i] < g.cand_ms[best]) best = i;
        const std::pair<int, int> choice = g.cands[best];
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[g.tune_key] = choice;
        }
        g.cands.clear();
        g.cand_ms.clear();
        drop_graph(b);
        if (!layout_group(b, g, choice.first, choice.second)) layout_group(b, g, choice.first, default_tps(g, choice.first));
        CU(cudaMemcpyAsync((unsigned char*)b->gmem + g.off_d, b->hbuf.data() + g.off_d, g.tab_bytes,
                           cudaMemcpyHostToDevice, b->stream));
    }
    return VFPS_OK;
}

// Queue k steps of every group: each group stream waits for the batch
// stream (fork), runs its k launches, and the batch stream waits for all of
// them again (join).  With timing, a group under tuning gets the layout of
// its candidate and start/stop events around its launches.
int enqueue_steps(vfps_batch* b, long long k, bool timing)
{
    cudaEvent_t fork = b->events.back();
    CU(cudaEventRecord(fork, b->stream));
    for (const Group& g : b->groups) CU(cudaStreamWaitEvent(g.stream, fork, 0));
    for (Group& g : b->groups) {
        if (!timing || g.cands.empty()) continue;
        if (g.cand >= 0) {  // upload the layout of the candidate under test
            const int cw = g.cands[g.cand].first;
            if (!layout_group(b, g, cw, g.cands[g.cand].second)) layout_group(b, g, cw, default_tps(g, cw));
            CU(cudaMemcpyAsync((unsigned char*)b->gmem + g.off_d, b->hbuf.data() + g.off_d, g.tab_bytes,
                               cudaMemcpyHostToDevice, g.stream));
        }
        CU(cudaEventRecord(g.t0, g.stream));
    }
    for (long long s = 0; s < k; ++s)
        for (const Group& g : b->groups) {
            const int rc = launch_step(g, g.stream);
            if (rc) return rc;
        }
    for (size_t i = 0; i < b->groups.size(); ++i) {
        if (timing && !b->groups[i].cands.empty()) CU(cudaEventRecord(b->groups[i].t1, b->groups[i].stream));
        CU(cudaEventRecord(b->events[i], b->groups[i].stream));
        CU(cudaStreamWaitEvent(b->stream, b->events[i], 0));
    }
    return VFPS_OK;
}

// Capture kGraphSteps steps of the current layout (no group under tuning)
// into the batch's graph, once per layout.
int ensure_batch_graph(vfps_batch* b)
{
    if (b->graph) return VFPS_OK;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_steps(b, kGraphSteps, false);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) {
        note_cuda_error(e, "cudaStreamEndCapture (batch)");
        return VFPS_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        b->graph = nullptr;
        note_cuda_error(ei, "cudaGraphInstantiate (batch)");
        return VFPS_ECUDA;
    }
    return VFPS_OK;
}

}  // namespace

extern "C" {

int64_t vfps_batch_slot_bytes(const vfps_params* params)
{
    if (check_params(params)) return -1;
    size_t offs[kInstanceSlots];
    return (int64_t)instance_bytes(params, kRingDefault / 2, offs);
}

int vfps_batch_create(int32_t max_slots, int64_t budget_bytes, void* cuda_stream, vfps_batch** out)
{
    if (!out || max_slots < 1 || budget_bytes < 0) return VFPS_EINVAL;
    *out = nullptr;
    std::unique_ptr<vfps_batch> b(new (std::nothrow) vfps_batch());
    if (!b) return VFPS_ENOMEM;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        CU(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    b->max_slots = max_slots;
    b->budget = budget_bytes;
    b->slots.assign(max_slots, nullptr);
    *out = b.release();
    return VFPS_OK;
}

int vfps_batch_add(vfps_batch* b, const vfps_params* params, const double* psi0, int model, double Pi,
                   double S_csr, const double* table, int64_t nsteps, int32_t* slot)
{
    if (!b || !slot || nsteps < 0) return VFPS_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    int free_slot = -1;
    for (int i = 0; i < b->max_slots; ++i)
        if (!b->slots[i]) {
            free_slot = i;
            break;
        }
    if (free_slot < 0) return VFPS_EBUSY;
    size_t offs[kInstanceSlots];
    long long need = (long long)instance_bytes(params, kRingDefault / 2, offs);
    if (b->budget > 0 && b->used + need > b->budget) return VFPS_EBUSY;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (long long)fr < need + (64ll << 20)) return VFPS_EBUSY;
    rc = init_kernels();
    if (rc) return rc;
    if (!b->adm) {
        CU(cudaStreamCreateWithFlags(&b->adm, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&b->adm_ev, cudaEventDisableTiming));
    }
    Instance* I = nullptr;
    rc = create_instance(params, psi0, kRingDefault / 2, b->adm, &I);
    if (rc) return rc;
    I->target = nsteps;
    rc = upload_impedance(*I, model, Pi, S_csr, table, b->adm);
    if (rc == VFPS_OK) rc = prologue(*I, b->adm);
    if (rc == VFPS_OK && (cudaEventRecord(b->adm_ev, b->adm) != cudaSuccess ||
                          cudaStreamWaitEvent(b->stream, b->adm_ev, 0) != cudaSuccess))
        rc = VFPS_ECUDA;
    if (rc) {
        cudaStreamSynchronize(b->adm);
        destroy_instance(I);
        return rc;
    }
    b->slots[free_slot] = I;
    b->used += (long long)I->dbytes;
    b->dirty = true;
    *slot = free_slot;
    return VFPS_OK;
}

int vfps_batch_run(vfps_batch* b, int64_t chunk_steps)
{
    if (!b || chunk_steps < 0) return VFPS_EINVAL;
    Range r("vfps_batch_run");
    int rc;
    while (chunk_steps > 0) {
        if (b->dirty) {
            rc = rebuild_groups(b);
            if (rc) return rc;
        }
        // steps until the next slot finishes or a ring fills
        long long k = chunk_steps;
        bool any = false;
        for (Instance* I : b->slots) {
            if (!I || remaining(I) <= 0) continue;
            any = true;
            k = std::min(k, remaining(I));
            long long room = (long long)I->ring - 1 - (I->steps_queued - I->drained);
            if (room <= 0) {
                rc = drain(*I, b->stream);
                if (rc) return rc;
                room = (long long)I->ring - 1;
            }
            k = std::min(k, room);
        }
        if (!any) break;
        // while a group is being tuned, kTuneSteps steps at a time (back to
        // back, as in steady state), timed on the group's own stream with the
        // candidate under test
        bool tuning = false;
        for (const Group& g : b->groups) tuning = tuning || !g.cands.empty();
        if (tuning) k = std::min<long long>(k, kTuneSteps);
        if (!tuning && k >= kGraphSteps) {
            // whole graphs of kGraphSteps steps: one host call per graph
            // instead of a fork, a launch per group and step, and a join
            rc = ensure_batch_graph(b);
            if (rc) return rc;
            const long long ng = k / kGraphSteps;
            for (long long i = 0; i < ng; ++i) CU(cudaGraphLaunch(b->graph, b->stream));
            k = ng * kGraphSteps;
        } else {
            rc = enqueue_steps(b, k, true);
            if (rc) return rc;
        }
        if (tuning) {
            rc = tune_step_done(b);
            if (rc) return rc;
        }
        for (Instance* I : b->slots) {
            if (!I || remaining(I) <= 0) continue;
            I->steps_queued += k;
            if (remaining(I) == 0) b->dirty = true;
        }
        chunk_steps -= k;
    }
    return VFPS_OK;
}

int vfps_batch_add_many(vfps_batch* b, int32_t count, const vfps_params* params, const double* psi0, int model,
                        const double* Pi, const double* S_csr, int64_t nsteps, int32_t* slots)
{
    if (!b || count < 1 || !Pi || !S_csr || !slots || nsteps < 0 || model < 0 || model > 2) return VFPS_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    std::vector<int> free_slots;
    for (int i = 0; i < b->max_slots && (int)free_slots.size() < count; ++i)
        if (!b->slots[i]) free_slots.push_back(i);
    if ((int)free_slots.size() < count) return VFPS_EBUSY;
    size_t offs[kInstanceSlots];
    const long long need = (long long)instance_bytes(params, kRingDefault / 2, offs) * count;
    if (b->budget > 0 && b->used + need > b->budget) return VFPS_EBUSY;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (long long)fr < need + (64ll << 20)) return VFPS_EBUSY;
    for (int i = 0; i < count; ++i)
        if ((model == 2 && !(Pi[i] > 0.0)) || !std::isfinite(S_csr[i])) return VFPS_EINVAL;
    rc = init_kernels();
    if (rc) return rc;
    if (!b->adm) {
        CU(cudaStreamCreateWithFlags(&b->adm, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&b->adm_ev, cudaEventDisableTiming));
    }
    std::vector<Instance*> made;
    auto fail = [&](int code) {
        cudaStreamSynchronize(b->adm);
        for (Instance* I : made) destroy_instance(I);
        return code;
    };
    // one allocation for all the slots (freed with the last of them)
    const size_t stride = align_up(instance_bytes(params, kRingDefault / 2, offs), kAlign);
    void* block = nullptr;
    if (dev_alloc(&block, stride * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        return VFPS_ENOMEM;
    }
    std::shared_ptr<void> arena(block, [](void* q) { cudaFree(q); });
    CU(cudaMemsetAsync(block, 0, stride * (size_t)count, b->adm));
    for (int i = 0; i < count; ++i) {
        Instance* I = nullptr;
        rc = create_instance(params, nullptr, kRingDefault / 2, b->adm, &I, false, false, false, arena,
                             stride * (size_t)i);
        if (rc) return fail(rc);
        I->target = nsteps;
        made.push_back(I);
    }
    arena.reset();  // the slots hold it now
    // every slot's tables in one host block, one copy, one scatter launch:
    // the twiddles, tile and segment lists and the state word are the same
    // for all slots (staged once), the impedance and descriptor per slot
    std::vector<unsigned char> img;
    std::vector<CopyJob> jobs;
    auto stage = [&](const void* src, size_t bytes) {
        const size_t off = align_up(img.size(), 16);
        img.resize(off + bytes);
        std::memcpy(img.data() + off, src, bytes);
        return off;
    };
    auto job = [&](size_t off, void* dst, size_t bytes) {
        jobs.push_back(CopyJob{(const unsigned int*)(uintptr_t)off, (unsigned int*)dst, (long long)(bytes / 4)});
    };
    {
        const Instance& I0 = *made[0];
        std::vector<unsigned char> tw;
        twiddle_table(I0, tw);
        std::vector<int2> t((size_t)I0.ntiles);
        std::vector<int4> sg((size_t)I0.ntiles);
        for (int k = 0; k < I0.ntiles; ++k) {
            t[(size_t)k] = make_int2(0, k * I0.W);
            sg[(size_t)k] = make_int4(0, k * I0.W, 1, 0);
        }
        DevState st{};
        st.scale = 1.0;
        const size_t o_tw = stage(tw.data(), tw.size()), o_t = stage(t.data(), sizeof(int2) * t.size());
        const size_t o_sg = stage(sg.data(), sizeof(int4) * sg.size()), o_st = stage(&st, sizeof(st));
        std::vector<unsigned char> zb;
        for (int i = 0; i < count && rc == VFPS_OK; ++i) {
            Instance& I = *made[(size_t)i];
            rc = impedance_image(I, model, Pi[i], S_csr[i], nullptr, zb);
            if (rc) break;
            if (I.p.precision) fill_desc<double>(I);
            else fill_desc<float>(I);
            job(o_tw, I.tw, tw.size());
            job(o_t, I.dtiles, sizeof(int2) * t.size());
            job(o_sg, I.dsegs, sizeof(int4) * sg.size());
            job(o_st, I.st, sizeof(st));
            job(stage(zb.data(), zb.size()), I.zhat, zb.size());
            job(stage(I.hdesc, sizeof(Desc<double>)), I.ddesc, sizeof(Desc<double>));
        }
    }
    // the prologue of every new slot (profile, wake and kick table of its
    // start) as one launch: their descriptors and tiles, staged with the rest
    const size_t dsz = params->precision ? sizeof(Desc<double>) : sizeof(Desc<float>);
    size_t o_descs = 0, o_tiles = 0;
    int ptiles = 0;
    if (rc == VFPS_OK) {
        o_descs = align_up(img.size(), 256);
        img.resize(o_descs + dsz * (size_t)count);
        std::vector<int2> pt;
        for (int i = 0; i < count; ++i) {
            std::memcpy(img.data() + o_descs + dsz * (size_t)i, made[(size_t)i]->hdesc, dsz);
            for (int k = 0; k < made[(size_t)i]->ntiles; ++k) pt.push_back(make_int2(i, k * made[(size_t)i]->W));
        }
        ptiles = (int)pt.size();
        o_tiles = stage(pt.data(), sizeof(int2) * pt.size());
    }
    unsigned char* dstage = nullptr;
    if (rc == VFPS_OK) {
        const size_t jo = align_up(img.size(), kAlign);
        unsigned char* d = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&d, jo + sizeof(CopyJob) * jobs.size(), b->adm);
        if (e == cudaSuccess) {
            for (CopyJob& j : jobs) j.src = (const unsigned int*)(d + (uintptr_t)j.src);
            e = cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, b->adm);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d + jo, jobs.data(), sizeof(CopyJob) * jobs.size(), cudaMemcpyHostToDevice, b->adm);
            if (e == cudaSuccess) {
                scatter_kernel<<<(unsigned)jobs.size(), 128, 0, b->adm>>>((const CopyJob*)(d + jo));
                e = cudaGetLastError();
            }
            dstage = d;
        }
        if (e != cudaSuccess) {
            note_cuda_error(e, "vfps_batch_add_many tables");
            rc = VFPS_ECUDA;
        }
    }
    if (rc == VFPS_OK) rc = upload_states(made.data(), count, psi0, b->adm);
    if (rc == VFPS_OK) {
        Group g = single_group(*made[0]);
        g.ddescs = dstage + o_descs;
        g.dtiles = (int2*)(dstage + o_tiles);
        g.ntiles = g.grid = ptiles;
        rc = launch_project(g, b->adm);
    }
    if (dstage) cudaFreeAsync(dstage, b->adm);
    if (rc == VFPS_OK && (cudaEventRecord(b->adm_ev, b->adm) != cudaSuccess ||
                          cudaStreamWaitEvent(b->stream, b->adm_ev, 0) != cudaSuccess))
        rc = VFPS_ECUDA;
    if (rc) return fail(rc);
    for (int i = 0; i < count; ++i) {
        b->slots[(size_t)free_slots[(size_t)i]] = made[(size_t)i];
        b->used += (long long)made[(size_t)i]->dbytes;
        slots[i] = free_slots[(size_t)i];
    }
    b->dirty = true;
    return VFPS_OK;
}

}  // extern "C"

namespace {

// Queue the gather of the states of one precision among inst (FP64 values
// at off[i] of the staged block d); the job table goes to d + job_off.
template <typename T>
int take_states_t(std::vector<Instance*>& inst, const std::vector<long long>& off, unsigned char* d,
                  size_t job_off, cudaStream_t s)
{
    std::vector<StateJob<T>> jobs;
    for (size_t i = 0; i < inst.size(); ++i) {
        const Instance& I = *inst[i];
        if ((I.p.precision != 0) != (sizeof(T) == 8)) continue;
        jobs.push_back(StateJob<T>{{(T*)I.psi[0], (T*)I.psi[1]}, I.st, off[i], 0.0, I.n, I.ld});
    }
    if (jobs.empty()) return VFPS_OK;
    StateJob<T>* dj = (StateJob<T>*)(d + job_off);
    CU(cudaMemcpyAsync(dj, jobs.data(), sizeof(StateJob<T>) * jobs.size(), cudaMemcpyHostToDevice, s));
    const int rows = stage_rows(jobs[0].n, (int)jobs.size());
    stage_load_kernel<T><<<dim3((unsigned)rows, (unsigned)jobs.size()), 256, 0, s>>>((double*)d, dj);
    CU(cudaGetLastError());
    return VFPS_OK;
}

}  // namespace

extern "C" {

int vfps_batch_take_many(vfps_batch* b, int32_t count, const int32_t* slots, double* psi_out, double* power_out,
                         int64_t power_cap, int64_t* n_power)
{
    if (!b || count < 1 || !slots || power_cap < 0 || (power_out && power_cap > 0 && !n_power)) return VFPS_EINVAL;
    std::vector<Instance*> inst((size_t)count);
    std::vector<long long> off((size_t)count);
    long long total = 0, kmax = 0;
    for (int i = 0; i < count; ++i) {
        const int sl = slots[i];
        if (sl < 0 || sl >= b->max_slots || !b->slots[(size_t)sl]) return VFPS_EINVAL;
        Instance* I = b->slots[(size_t)sl];
        inst[(size_t)i] = I;
        off[(size_t)i] = total;
        total += (long long)I->n * I->n;
        kmax = std::max(kmax, I->steps_queued - I->drained);
    }
    // staged block: states (FP64), the undrained ring entries of every state
    // (kmax per row), the status words, then the job tables
    const size_t vb = align_up((size_t)total * 8, kAlign);
    const size_t pb = align_up((size_t)count * 2 * (size_t)std::max<long long>(kmax, 1) * 8, kAlign);
    const size_t stb = align_up((size_t)count * 4, kAlign);
    const size_t jb = align_up(sizeof(SeriesJob) * (size_t)count, kAlign);
    const size_t tjb = sizeof(StateJob<double>) * (size_t)count;
    unsigned char* d = nullptr;
    CU(cudaMallocAsync((void**)&d, vb + pb + stb + jb + 2 * tjb, b->stream));
    std::vector<SeriesJob> sj((size_t)count);
    for (int i = 0; i < count; ++i) {
        const Instance& I = *inst[(size_t)i];
        sj[(size_t)i] = SeriesJob{I.pring, I.qring, I.st, I.drained, I.steps_queued - I.drained, (long long)I.ring - 1};
    }
    std::vector<double> series((size_t)count * 2 * (size_t)std::max<long long>(kmax, 1));
    std::vector<int> status((size_t)count);
    int rc = VFPS_OK;
    cudaError_t e = cudaMemcpyAsync(d + vb + pb + stb, sj.data(), sizeof(SeriesJob) * sj.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && psi_out) {
        rc = take_states_t<float>(inst, off, d, vb + pb + stb + jb, b->stream);
        if (rc == VFPS_OK) rc = take_states_t<double>(inst, off, d, vb + pb + stb + jb + tjb, b->stream);
    }
    if (e == cudaSuccess && rc == VFPS_OK) {
        stage_series_kernel<<<count, 256, 0, b->stream>>>((double*)(d + vb), std::max<long long>(kmax, 1),
                                                          (const SeriesJob*)(d + vb + pb + stb), (int*)(d + vb + pb));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == VFPS_OK && psi_out)
        e = cudaMemcpyAsync(psi_out, d, (size_t)total * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && rc == VFPS_OK)
        e = cudaMemcpyAsync(series.data(), d + vb, series.size() * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && rc == VFPS_OK)
        e = cudaMemcpyAsync(status.data(), d + vb + pb, status.size() * 4, cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(d, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        note_cuda_error(e, "vfps_batch_take_many");
        return VFPS_ECUDA;
    }
    if (rc) return rc;
    for (int i = 0; i < count; ++i) {
        Instance& I = *inst[(size_t)i];
        const size_t cap = (size_t)std::max<long long>(kmax, 1);
        const double* rp = series.data() + (size_t)(2 * i) * cap;
        I.pw.insert(I.pw.end(), rp, rp + sj[(size_t)i].cnt);
        I.qw.insert(I.qw.end(), rp + cap, rp + cap + sj[(size_t)i].cnt);
        I.drained = I.steps_queued;
        rc = drain_moments(I, b->stream);
        if (rc) return rc;
        if (power_out && power_cap > 0) {
            const int64_t k = std::min<int64_t>(power_cap, (int64_t)I.pw.size());
            std::memcpy(power_out + (size_t)i * (size_t)power_cap, I.pw.data(), sizeof(double) * (size_t)k);
            n_power[i] = k;
        }
    }
    for (int i = 0; i < count; ++i) {
        rc = status_code(status[(size_t)i]);
        if (rc) return rc;
    }
    return VFPS_OK;
}

int vfps_batch_idle(vfps_batch* b, int32_t* idle)
{
    if (!b || !idle) return VFPS_EINVAL;
    const cudaError_t e = cudaStreamQuery(b->stream);
    if (e == cudaErrorNotReady) {
        *idle = 0;
        return VFPS_OK;
    }
    CU(e);
    *idle = 1;
    return VFPS_OK;
}

int vfps_batch_poll(vfps_batch* b, int32_t* done_slots, int32_t cap, int32_t* n_done)
{
    if (!b || !n_done || cap < 0 || (cap > 0 && !done_slots)) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(b->stream));
    int k = 0;
    for (int i = 0; i < b->max_slots; ++i) {
        Instance* I = b->slots[i];
        if (I && remaining(I) <= 0) {
            if (k < cap) done_slots[k] = i;
            ++k;
        }
    }
    *n_done = std::min(k, cap);
    return VFPS_OK;
}

int vfps_batch_take(vfps_batch* b, int32_t slot, double* psi_out, double* rho_out, double* power_out,
                    int64_t power_cap, int64_t* n_power, int64_t* steps_done)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return VFPS_EINVAL;
    Instance& I = *b->slots[slot];
    int rc = drain(I, b->stream);
    if (rc) return rc;
    if (psi_out) {
        rc = copy_state(I, b->stream, psi_out);
        if (rc) return rc;
    }
    if (rho_out) CU(cudaMemcpyAsync(rho_out, I.rho, sizeof(double) * I.n, cudaMemcpyDeviceToHost, b->stream));
    if (power_out && power_cap > 0) {
        int64_t k = std::min<int64_t>(power_cap, (int64_t)I.pw.size());
        std::memcpy(power_out, I.pw.data(), sizeof(double) * k);
        if (n_power) *n_power = k;
    } else if (n_power) {
        *n_power = (int64_t)I.pw.size();
    }
    if (steps_done) *steps_done = I.steps_queued;
    // copy_state has already synchronised and read the status word; rho (if
    // asked for) still needs a synchronisation, read_status provides it
    if (psi_out && !rho_out) return VFPS_OK;
    return read_status(I, b->stream);
}

int vfps_batch_shapes(vfps_batch* b, int32_t* out, int32_t cap, int32_t* n_groups)
{
    if (!b || !n_groups || cap < 0 || (cap > 0 && !out)) return VFPS_EINVAL;
    if (b->dirty) {
        int rc = rebuild_groups(b);
        if (rc) return rc;
    }
    int k = 0;
    for (const Group& g : b->groups) {
        if (k < cap) {
            out[6 * k] = g.n;
            out[6 * k + 1] = (int32_t)g.members.size();
            out[6 * k + 2] = g.W;
            out[6 * k + 3] = g.tps;
            out[6 * k + 4] = g.cands.empty() ? 1 : 0;
            out[6 * k + 5] = g.pair;
        }
        ++k;
    }
    *n_groups = std::min(k, cap);
    return VFPS_OK;
}

int vfps_batch_pairing(vfps_batch* b, int32_t on)
{
    if (!b || (on != 0 && on != 1)) return VFPS_EINVAL;
    b->pairing = on != 0;
    b->dirty = true;
    return VFPS_OK;
}

int vfps_batch_pin_shape(vfps_batch* b, int32_t W, int32_t tps)
{
    if (!b || !((W == 0 && tps == 0) || ((W == 2 || W == 4 || W == 8) && ((tps >= 1 && tps <= 256) || tps == -1))))
        return VFPS_EINVAL;
    b->pin_W = W;
    b->pin_tps = tps;
    b->dirty = true;
    return VFPS_OK;
}

int vfps_batch_autotune(vfps_batch* b, int32_t on)
{
    if (!b || (on != 0 && on != 1)) return VFPS_EINVAL;
    b->autotune = on == 1;
    return VFPS_OK;
}

int vfps_batch_power_spectrum(vfps_batch* b, int32_t slot, int32_t length, double* out)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return VFPS_EINVAL;
    return instance_power_spectrum(*b->slots[slot], b->stream, length, out);
}

int vfps_batch_moments(vfps_batch* b, int32_t slot, double* out)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return VFPS_EINVAL;
    return instance_moments(*b->slots[slot], b->stream, out);
}

int vfps_batch_record_moments(vfps_batch* b, int32_t slot, int32_t every)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot] || every < 0) return VFPS_EINVAL;
    Instance& I = *b->slots[slot];
    const bool had = I.mring != nullptr;
    CU(cudaStreamSynchronize(b->stream));
    const int rc = set_moment_recording(I, b->stream, every);
    if (rc) return rc;
    if (!had && I.mring) b->used += (long long)(sizeof(double) * 4 * (size_t)I.ring);
    b->dirty = true;  // the launch groups hold copies of the descriptor
    return VFPS_OK;
}

int vfps_batch_moment_series(vfps_batch* b, int32_t slot, double* out, int64_t cap, int64_t* n_written)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot] || !n_written || cap < 0 || (cap > 0 && !out))
        return VFPS_EINVAL;
    Instance& I = *b->slots[slot];
    int rc = drain(I, b->stream);
    if (rc) return rc;
    *n_written = take_moments(I, out, cap, false);
    return read_status(I, b->stream);
}

int vfps_batch_spectrogram(vfps_batch* b, const int32_t* slots, int32_t nslots, int32_t length, int32_t hop,
                           int32_t count, double* out)
{
    if (!b || !slots || nslots < 1) return VFPS_EINVAL;
    std::vector<Instance*> inst((size_t)nslots);
    for (int i = 0; i < nslots; ++i) {
        const int sl = slots[i];
        if (sl < 0 || sl >= b->max_slots || !b->slots[sl]) return VFPS_EINVAL;
        inst[(size_t)i] = b->slots[sl];
    }
    return spectrogram(inst.data(), nslots, length, hop, count, b->stream, out);
}

int vfps_batch_haissinski(vfps_batch* b, int32_t slot, double tol, int32_t max_iter, int32_t* iterations)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(b->stream));
    return instance_haissinski(*b->slots[slot], b->stream, tol, max_iter, iterations);
}

int vfps_batch_remove(vfps_batch* b, int32_t slot)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return VFPS_EINVAL;
    CU(cudaStreamSynchronize(b->stream));
    b->used -= (long long)b->slots[slot]->dbytes;
    if (b->slots[slot]->mring) b->used -= (long long)(sizeof(double) * 4 * (size_t)b->slots[slot]->ring);
    destroy_instance(b->slots[slot]);
    b->slots[slot] = nullptr;
    b->dirty = true;
    return VFPS_OK;
}

int vfps_batch_launches_per_step(vfps_batch* b, int32_t* launches)
{
    if (!b || !launches) return VFPS_EINVAL;
    if (b->dirty) {
        int rc = rebuild_groups(b);
        if (rc) return rc;
    }
    *launches = (int32_t)b->groups.size();
    return VFPS_OK;
}

int vfps_batch_usage(vfps_batch* b, int32_t* active, int64_t* bytes)
{
    if (!b) return VFPS_EINVAL;
    int k = 0;
    for (Instance* I : b->slots)
        if (I) ++k;
    if (active) *active = k;
    if (bytes) *bytes = b->used;
    return VFPS_OK;
}

int vfps_batch_destroy(vfps_batch* b)
{
    if (!b) return VFPS_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (cudaStream_t st : b->pool) cudaStreamSynchronize(st);
    for (Instance* I : b->slots) destroy_instance(I);
    free_groups(b);
    for (cudaStream_t st : b->pool) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->events) cudaEventDestroy(ev);
    if (b->adm) {
        cudaStreamSynchronize(b->adm);
        cudaStreamDestroy(b->adm);
        cudaEventDestroy(b->adm_ev);
    }
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return VFPS_OK;
}

}  // extern "C"

// ============================================================================
// Allocation-free single step (vfps_step_static).
//
// Some callers may not allocate device memory at all: plug-ins living inside
// a host application whose memory pool owns the whole device (an allocation
// behind the pool's back can fail or fragment it), and latency-critical loops
// that cannot afford cudaMalloc's implicit synchronisation or its failure
// path.  This entry point advances one caller-owned FP32 state by one step
// using only the caller's buffers and a fixed scratch area that lives in the
// library image itself, so it never calls cudaMalloc or cudaFree.
//
// Scratch: g_vfps_static_scratch below (STATIC_SCRATCH_BYTES, about 80 KB),
// sized for n <= 1024 and an FFT length M <= 4096.  Every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps
// the last call's contents; each call rewrites the parts that must start
// fresh (descriptor, tile list, state word with its zero ticket, impedance,
// twiddles), and the column sums, profile and kick are fully overwritten by
// the kernels before they are read.  Calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on this scratch.
namespace {

constexpr int kStaticMaxN = 1024;
constexpr int kStaticMaxFFT = 4096;
constexpr size_t kSA = 256;
constexpr size_t sa(size_t v) { return (v + kSA - 1) / kSA * kSA; }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffTiles = kOffDesc + sa(sizeof(Desc<float>));
constexpr size_t kOffSegs = kOffTiles + sa(sizeof(int2) * (kStaticMaxN / 2 + 1));
constexpr size_t kOffState = kOffSegs + sa(sizeof(int4) * (kStaticMaxN / 2 + 1));
constexpr size_t kOffColsum = kOffState + sa(sizeof(DevState));
constexpr size_t kOffRho = kOffColsum + sa(sizeof(double) * kStaticMaxN);
constexpr size_t kOffKick = kOffRho + sa(sizeof(double) * kStaticMaxN);
constexpr size_t kOffKickW = kOffKick + sa(sizeof(float) * kStaticMaxN);
constexpr size_t kOffZhat = kOffKickW + sa(2 * sizeof(float4) * kStaticMaxN);
constexpr size_t kOffTw = kOffZhat + sa(sizeof(float2) * (kStaticMaxFFT / 2 + 1));
constexpr size_t kOffRings = kOffTw + sa(sizeof(float2) * (kStaticMaxFFT / 2));
constexpr size_t STATIC_SCRATCH_BYTES = kOffRings + sa(sizeof(double) * 4);

}  // namespace

static __device__ __align__(256) unsigned char g_vfps_static_scratch[STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
void* g_static_dev_ptr[64] = {};
// host-side staging of what each call uploads (guarded by g_static_mu)
unsigned char g_static_host[kOffRings];

// Device address of the scratch on the current device.  In host code the
// array's name only stands in for it, so it is looked up once per device
// (with that device current) and cached.
int static_scratch(void** out)
{
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return VFPS_EINVAL;
    if (!g_static_dev_ptr[dev]) {
        void* p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_vfps_static_scratch));
        g_static_dev_ptr[dev] = p;
    }
    *out = g_static_dev_ptr[dev];
    return VFPS_OK;
}

__global__ void static_scale_kernel(float* psi, int n, const DevState* st)
{
    const float s = float(st->scale);
    const size_t nn = (size_t)n * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        psi[i] *= s;
}

int static_fail(const char* msg)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    return VFPS_EINVAL;
}

}  // namespace

extern "C" int vfps_step_static(const vfps_params* params, int model, double Pi, double S_csr,
                                const float* psi_in, float* psi_out, double* power_out, void* cuda_stream)
{
    int rc = check_params(params);
    if (rc) return static_fail("vfps_step_static: invalid parameters");
    if (params->precision != 0) return static_fail("vfps_step_static: FP32 states only (precision = 0)");
    if (params->n > kStaticMaxN) {
        char m[160];
        std::snprintf(m, sizeof(m), "vfps_step_static: n = %d exceeds the static scratch limit of %d points per axis",
                      params->n, kStaticMaxN);
        return static_fail(m);
    }
    const int M = fft_length(params);
    if (M > kStaticMaxFFT) {
        char m[160];
        std::snprintf(m, sizeof(m), "vfps_step_static: FFT length %d exceeds the static scratch limit of %d", M,
                      kStaticMaxFFT);
        return static_fail(m);
    }
    if (!psi_in || !psi_out || psi_in == (const float*)psi_out)
        return static_fail("vfps_step_static: psi_in and psi_out must be two distinct device buffers");
    if (model < 0 || model > 2 || (model == 2 && !(Pi > 0.0)) || !std::isfinite(S_csr))
        return static_fail("vfps_step_static: impedance model 0, 1 or 2 (Pi > 0) and a finite S_csr");
    int fast = 0;
    const int W = choose_width(params, &fast, true);
    if (W == 0) return static_fail("vfps_step_static: grid too large for the staged slab at this step angle");
    if (fast && (((uintptr_t)psi_in | (uintptr_t)psi_out) & 15))
        return static_fail("vfps_step_static: psi buffers must be 16-byte aligned");
    rc = init_kernels();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> lock(g_static_mu);
    void* base = nullptr;
    rc = static_scratch(&base);
    if (rc) return rc;
    unsigned char* d = (unsigned char*)base;

    // the simulation's buffers: caller's psi, scratch for everything else
    Instance I;
    I.p = *params;
    I.p.renormalize = 1;  // psi_out is normalised to charge 1 whatever the caller's flag
    I.n = params->n;
    I.ld = params->n;
    I.M = M;
    I.W = W;
    I.fast = fast;
    I.ntiles = (params->n + W - 1) / W;
    I.ring = 2;
    I.delta = 2.0 * params->half_width / (params->n - 1);
    I.phi = 2.0 * kPi / params->steps_per_period;
    I.S = S_csr;
    I.psi[0] = (void*)psi_in;
    I.psi[1] = psi_out;
    I.zhat = d + kOffZhat;
    I.tw = d + kOffTw;
    I.colsum = (double*)(d + kOffColsum);
    I.rho = (double*)(d + kOffRho);
    I.kick = d + kOffKick;
    I.kickw = d + kOffKickW;
    I.pring = (double*)(d + kOffRings);
    I.qring = (double*)(d + kOffRings) + 2;
    I.st = (DevState*)(d + kOffState);
    fill_desc<float>(I);

    // stage the per-call inputs on the host, then upload them
    unsigned char* h = g_static_host;
    std::memcpy(h + kOffDesc, I.hdesc, sizeof(Desc<float>));
    int2* tiles = (int2*)(h + kOffTiles);
    int4* segs = (int4*)(h + kOffSegs);
    for (int i = 0; i < I.ntiles; ++i) {
        tiles[i] = make_int2(0, i * W);
        segs[i] = make_int4(0, i * W, 1, 0);
    }
    DevState st{};
    st.scale = 1.0;
    std::memcpy(h + kOffState, &st, sizeof(st));
    std::vector<std::complex<double>> z;
    cached_impedance(model, M, I.delta, Pi, z);
    float2* zh = (float2*)(h + kOffZhat);
    for (int k = 0; k <= M / 2; ++k) zh[k] = make_float2((float)z[k].real(), (float)z[k].imag());
    float2* tw = (float2*)(h + kOffTw);
    for (int k = 0; k < M / 2; ++k) {
        const double ang = -2.0 * kPi * k / M;
        tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    CU(cudaMemcpyAsync(d, h, kOffRings, cudaMemcpyHostToDevice, s));

    Group g;
    g.prec = 0;
    g.ni = params->interp_points;
    g.W = W;
    g.fast = fast;
    g.var = !fast ? 0 : (params->clamp ? 2 : (params->interp_points != 4 ? 1 : 0));
    g.kr = fast_kr(params->n);
    g.n = params->n;
    g.rot = params->rotation;
    g.ntiles = I.ntiles;
    g.smem = fast ? std::max(fast_smem(params, W), step_smem(params, W)) : step_smem(params, W);
    g.ddescs = d + kOffDesc;
    g.dtiles = (int2*)(d + kOffTiles);
    g.dsegs = (int4*)(d + kOffSegs);
    g.grid = I.ntiles;
    rc = launch_project(g, s);   // profile, wake and P of psi_in
    if (rc) return rc;
    rc = launch_step(g, s);      // psi_out = one un-normalised step
    if (rc) return rc;
    static_scale_kernel<<<std::min(1024, (I.n * I.n + 255) / 256), 256, 0, s>>>(psi_out, I.n, I.st);
    CU(cudaGetLastError());
    if (power_out) {
        DevState out{};
        CU(cudaMemcpyAsync(power_out, I.pring, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(&out, I.st, sizeof(out), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (out.status) return out.status;
    }
    return VFPS_OK;
}

// C ABI of libmithra: run set-up (rest frame, mesh checks, placement), device memory,
// the per-step launch sequence and the accessors declared in include/mithra.h.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mithra.h"
#include "common.cuh"
#include "kernels.h"
#include "run.h"

using namespace mithra;

// ---------------------------------------------------------------------------------------
// errors and the allocator hook
// ---------------------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CU(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(MITHRA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Allocator {
    mithra_alloc_fn alloc = nullptr;
    mithra_free_fn free_fn = nullptr;
    void* ctx = nullptr;
};
static std::mutex g_alloc_mu;
static Allocator g_alloc;

extern "C" int mithra_set_allocator(mithra_alloc_fn alloc, mithra_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(MITHRA_EINVAL, "allocator: give both functions or none");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_fn = free_fn;
    g_alloc.ctx = ctx;
    return MITHRA_OK;
}

static std::atomic<int64_t> g_launches{0};
static thread_local int64_t t_launches = 0;   // this thread's launches (graph capture counts its nodes)
void mithra::count_launches(int64_t n)
{
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}
static int64_t launch_count() { return t_launches; }

// Block partials of the run's reductions: enough blocks of 256 threads to fill the GPU (8 on each of
// its 152 SMs), and one per 256 nodes of the power plane.
constexpr int kMinPartials = 1216;
static int run_partials(int64_t plane) { return std::max<int>(kMinPartials, (int)((plane + 255) / 256)); }
extern "C" int64_t mithra_kernel_launches(void) { return g_launches.load(); }

extern "C" const char* mithra_last_error(void) { return g_err.c_str(); }

void mithra::get_allocator(mithra_alloc_fn* alloc, mithra_free_fn* free_fn, void** ctx)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    *alloc = g_alloc.alloc;
    *free_fn = g_alloc.free_fn;
    *ctx = g_alloc.ctx;
}
int mithra::set_last_error(int code, const char* msg) { return fail(code, msg); }
extern "C" int mithra_version(void) { return 1; }

static const char* kKernelNames[MITHRA_K_COUNT] = {"emit_eb", "push_deposit", "stencil", "mur", "power", "sort",
                                                   "clear_sources"};
extern "C" const char* mithra_kernel_name(int id)
{
    return (id >= 0 && id < MITHRA_K_COUNT) ? kKernelNames[id] : "unknown";
}

// ---------------------------------------------------------------------------------------
// the run
// ---------------------------------------------------------------------------------------
// Device memory of one run.  Every array starts on a 256-byte boundary: the tensor maps, the
// 16-byte vector atomics of the deposit flush and the vector loads rely on it.  cudaMalloc
// guarantees it; a caller-installed allocator may return any alignment, so its blocks are
// requested 256 bytes longer and aligned here (the original pointer is what gets freed).
// Without a caller's allocator the run first reserves one slab for its known arrays and hands
// them out of it (one cudaMalloc instead of some fifty: a third of the time to create the FEL
// run); what does not fit, and temporaries, take their own cudaMalloc.
struct DevMem {
    struct Block {
        void* p;      // the aligned pointer handed out
        size_t bytes; // bytes taken from the allocator
        void* raw;    // the pointer the allocator returned (null: part of the slab)
    };
    Allocator a;
    std::vector<Block> blocks;
    size_t total = 0;
    char* slab = nullptr;
    size_t slab_size = 0, slab_used = 0;
    void reserve(size_t bytes)
    {
        if (a.alloc || slab) return;
        bytes = (bytes + 255) & ~(size_t)255;
        if (cudaMalloc((void**)&slab, bytes) != cudaSuccess) {
            cudaGetLastError();
            slab = nullptr;
            return;
        }
        slab_size = bytes;
    }
    // temp: a block released soon (not taken from the slab)
    void* get(size_t bytes, bool temp = false)
    {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~(size_t)255;
        if (!temp && slab && slab_used + bytes <= slab_size) {
            void* p = slab + slab_used;
            slab_used += bytes;
            blocks.push_back(Block{p, bytes, nullptr});
            total += bytes;
            return p;
        }
        void* raw = nullptr;
        if (a.alloc) {
            bytes += 256;
            raw = a.alloc(a.ctx, bytes);
        } else if (cudaMalloc(&raw, bytes) != cudaSuccess) {
            cudaGetLastError();
            raw = nullptr;
        }
        if (!raw) return nullptr;
        void* p = (void*)(((uintptr_t)raw + 255) & ~(uintptr_t)255);
        blocks.push_back(Block{p, bytes, raw});
        total += bytes;
        return p;
    }
    void release(void* p)
    {
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i].p == p) {
                total -= blocks[i].bytes;
                if (!blocks[i].raw) {
                    // a slab block: its space is reused only if it was the last one handed out
                    if ((char*)p + blocks[i].bytes == slab + slab_used) slab_used -= blocks[i].bytes;
                } else if (a.free_fn) {
                    a.free_fn(a.ctx, blocks[i].raw);
                } else {
                    cudaFree(blocks[i].raw);
                }
                blocks.erase(blocks.begin() + (long)i);
                return;
            }
    }
    void release_all()
    {
        for (auto& b : blocks) {
            if (!b.raw) continue;
            if (a.free_fn) a.free_fn(a.ctx, b.raw);
            else cudaFree(b.raw);
        }
        if (slab) cudaFree(slab);
        slab = nullptr;
        slab_size = slab_used = 0;
        blocks.clear();
        total = 0;
    }
};

struct Derived {
    double g0, b0, dx, dy, dz, dt, dtb, A, x0, y0, z0, T0, omega_h, M, kp, z_ref, q, kstar, kb;
};

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

struct mithra_run {
    virtual ~mithra_run() {}
    virtual int step(int64_t n) = 0;
    virtual int fields(int which, int level, double* out, size_t cap) = 0;
    virtual int set_field(int which, int level, const double* in, size_t n) = 0;
    virtual int particles(double* out, size_t cap) = 0;
    virtual int set_particles(const double* in, size_t n) = 0;
    virtual int diag(double* fe, double* b3) = 0;
    virtual int series(int which, double* out, size_t cap, size_t* n_out) = 0;
    virtual int spectrum(double* h, double* p, size_t cap, size_t* n_steps) = 0;
    virtual int set_seed(const mithra_seed& s) = 0;
    virtual int bunch_samples(double* out, size_t cap_rows, size_t* n_rows) = 0;
    virtual int sync() = 0;
    virtual int64_t graph_steps() const = 0;
    virtual cudaGraph_t period_graph(int64_t steps_left) = 0;
    virtual void period_replayed() = 0;
    virtual void destroy_all() = 0;

    // common state
    Derived d;
    Geom g;
    ExtField ef;
    StencilCoef cf;
    int precision = 1;
    int mur_order = 2;
    int sort_every = 20;
    int64_t np = 0;
    int64_t nstep = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevMem mem;
    // profiling
    bool prof = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_free;
    double prof_ms[MITHRA_K_COUNT] = {0};
    int64_t prof_n[MITHRA_K_COUNT] = {0};

    cudaEvent_t ev_get()
    {
        if (!ev_free.empty()) {
            cudaEvent_t e = ev_free.back();
            ev_free.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void prof_collect()
    {
        for (auto& r : prof_pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                prof_ms[r.kid] += ms;
                prof_n[r.kid] += 1;
            } else {
                cudaGetLastError();
            }
            ev_free.push_back(r.a);
            ev_free.push_back(r.b);
        }
        prof_pending.clear();
    }
};

namespace {

template <typename real>
struct RunT final : mithra_run {
    real* pot[3][4] = {};      // ring of three time levels of A_x, A_y, A_z, phi
    int base = 0;              // pot[(base + 0) % 3] = level n, (base + 1) % 3 = level n+1
    real* src[4] = {};
    real* eb = nullptr;   // E, B at the nodes, interleaved (Fields6)
    Particles<real> P{}, T{};
    SortScratch ss{};
    double* ring = nullptr;
    double* acc = nullptr;      // running DFT accumulators of the power plane
    double* partial = nullptr;
    float2* btab = nullptr;   // bunching: the node planes' phases (FP32 path)
    int npartial = kMinPartials;
    double* ser_p = nullptr;
    double* ser_e = nullptr;
    int64_t ser_cap = 0;
    double* small = nullptr;   // 8 doubles of diagnostic output
    // radiated-power spectrum (nf = 0: off)
    int nf = 0, Mh = 1;
    std::vector<double> hk;
    double* spec_omega = nullptr;
    int* spec_M = nullptr;
    double* spec_scale = nullptr;
    double* spec_ring = nullptr;
    double* spec_acc = nullptr;
    double* spec_partial = nullptr;
    double* ser_s = nullptr;   // ser_cap x nf
    // seed through TF/SF planes (seed.type < 0: none)
    SeedField seed{-1};
    double* seed_buf = nullptr;   // the seed potential on z planes 1, 2 (2 components)
    // bunch sampling (bunch_every = 0: off)
    int bunch_every = 0;
    double bunch_shift_g = 1.0;
    double* bunch_partial = nullptr;
    double* ser_b = nullptr;   // rows(ser_cap) x 15
    double* rest_buf = nullptr;
    int64_t onaxis_id = 0;
    int* box[2] = {nullptr, nullptr};   // deposit boxes of alternate steps (deposit_box_words each)
    int* box_rec = nullptr;              // the push's per-block bounds (six ints per block of 128)
    double2* ptab[2] = {nullptr, nullptr};   // static-undulator phase tables, FP64 path (one per planar field)
    float4* ptab32[2] = {nullptr, nullptr};  // FP32-mixed path: phase and edge distances rounded to FP32
    float4* ptab32a = nullptr;               // FP32-mixed path, undulator array: module peak fields per plane
    TmaMaps* tma = nullptr;    // tensor maps of the TMA stencil (null: plain stencil)
    MurFaceCoef murc{};        // Mur face coefficients (the FP32 TMA stencil writes the x faces)
    int* err_word = nullptr;   // set by a kernel whose bounded wait expired
    int test_tma_skip = -1;    // failure tests: TMA stencil plane left uncopied (-1: none)
    unsigned* counters = nullptr;   // last-block counters (Mur edges, power), zero between launches
    StepDev* sd = nullptr;     // per-step values derived on the device from the step counter
    StepConst scst{};
    // captured steps: one graph of glen steps replayed from every aligned step
    static constexpr int64_t kGraphMaxSteps = 480;
    bool use_graphs = true;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t gtmpl = nullptr;   // the captured steps as a graph (a serving group embeds it)
    int64_t glen = 0;
    int64_t gnodes = 0;

    int lev(int k) const { return (base + k) % 3; }

    // Make the box read by the next emission cover every active cell (start, new particles).
    int full_box(int which)
    {
        std::vector<int> h(deposit_box_ints(g.nz));
        const int whole[6] = {1, 1, 1, g.nx - 3, g.ny - 3, g.nz - 3};
        for (int q = 0; q < 6; ++q) h[q] = whole[q];
        for (size_t q = 6; q < h.size(); q += 4) {
            h[q] = 1;
            h[q + 1] = 1;
            h[q + 2] = g.nx - 3;
            h[q + 3] = g.ny - 3;
        }
        CU(cudaMemcpyAsync(box[which], h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    // E and B of the last step over the whole interior: after a step the ring holds
    // A^{n+1} at lev(0) and the step's A^n still at lev(2).
    int emit_full()
    {
        if (nstep == 0) return MITHRA_OK;
        FieldLevels<real> L;
        for (int c = 0; c < 4; ++c) {
            L.n0[c] = pot[lev(2)][c];
            L.n1[c] = pot[lev(0)][c];
            L.out[c] = nullptr;
            L.src[c] = src[c];
        }
        Fields6<real> E6;
        E6.p = eb;
        EmitBox bx{nullptr, nullptr, -1, false};
        EmitMaps em;
        if (emit_maps(tma, lev(2), lev(0), &em)) bx.maps = &em;
        bx.err = err_word;
        CU(launch_emit<real>(L, E6, g, bx, stream));
        return MITHRA_OK;
    }

    int alloc_all()
    {
        const size_t cell = (size_t)g.ncell * sizeof(real);
        for (int l = 0; l < 3; ++l)
            for (int c = 0; c < 4; ++c)
                if (!(pot[l][c] = (real*)mem.get(cell))) return fail(MITHRA_ENOMEM, "device allocation failed (fields)");
        for (int c = 0; c < 4; ++c)
            if (!(src[c] = (real*)mem.get(cell))) return fail(MITHRA_ENOMEM, "device allocation failed (sources)");
        if (!(eb = (real*)mem.get(cell * kEBStride))) return fail(MITHRA_ENOMEM, "device allocation failed (E/B)");
        for (int l = 0; l < 3; ++l)
            for (int c = 0; c < 4; ++c) CU(cudaMemsetAsync(pot[l][c], 0, cell, stream));
        for (int c = 0; c < 4; ++c) CU(cudaMemsetAsync(src[c], 0, cell, stream));
        CU(cudaMemsetAsync(eb, 0, cell * kEBStride, stream));
        const int64_t n = np > 0 ? np : 1;
        for (Particles<real>* Q : {&P, &T}) {
            Q->ix = (int32_t*)mem.get(n * 4);
            Q->iy = (int32_t*)mem.get(n * 4);
            Q->iz = (int32_t*)mem.get(n * 4);
            Q->fx = (real*)mem.get(n * sizeof(real));
            Q->fy = (real*)mem.get(n * sizeof(real));
            Q->fz = (real*)mem.get(n * sizeof(real));
            Q->ux = (mom_t<real>*)mem.get(n * sizeof(mom_t<real>));
            Q->uy = (mom_t<real>*)mem.get(n * sizeof(mom_t<real>));
            Q->uz = (mom_t<real>*)mem.get(n * sizeof(mom_t<real>));
            Q->id = (int32_t*)mem.get(n * 4);
            if (!Q->ix || !Q->iy || !Q->iz || !Q->fx || !Q->fy || !Q->fz || !Q->ux || !Q->uy || !Q->uz || !Q->id)
                return fail(MITHRA_ENOMEM, "device allocation failed (particles)");
        }
        ss.nbins = g.ncell + 1;
        ss.key = (int32_t*)mem.get(n * 4);
        ss.perm = (int32_t*)mem.get(n * 4);
        ss.count = (int32_t*)mem.get((size_t)ss.nbins * 4);
        ss.offset = (int32_t*)mem.get((size_t)ss.nbins * 4);
        ss.blocksum = (int32_t*)mem.get(sort_scan_partials(ss.nbins) * 4);
        if (!ss.key || !ss.perm || !ss.count || !ss.offset || !ss.blocksum)
            return fail(MITHRA_ENOMEM, "device allocation failed (sort scratch)");
        const int M = (int)d.M;
        const size_t plane = (size_t)g.nx * g.ny;
        npartial = run_partials(plane);
        ring = (double*)mem.get((size_t)M * 4 * plane * 8);
        acc = (double*)mem.get((size_t)8 * plane * 8);
        partial = (double*)mem.get((size_t)4 * npartial * 8);   // energy: [0, n); bunching: [n, 3n)
        small = (double*)mem.get(8 * 8);
        if (sizeof(real) == 4) btab = (float2*)mem.get((size_t)g.nz * sizeof(float2));
        if (!ring || !acc || !partial || !small || (sizeof(real) == 4 && !btab))
            return fail(MITHRA_ENOMEM, "device allocation failed (diagnostics)");
        CU(cudaMemsetAsync(ring, 0, (size_t)M * 4 * plane * 8, stream));
        CU(cudaMemsetAsync(acc, 0, (size_t)8 * plane * 8, stream));
        if (nf > 0) {
            std::vector<double> om(nf), sc(nf);
            std::vector<int> Mv(nf);
            const double f = d.g0 * d.g0 * (1.0 + d.b0) * (1.0 + d.b0);
            Mh = 1;
            for (int k = 0; k < nf; ++k) {
                om[k] = hk[k] * kC * d.kstar;
                double Mk = std::round(2.0 * kPi / (om[k] * d.dt));
                if (!(Mk >= 1.0)) Mk = 1.0;
                if (Mk > 1e6) return fail(MITHRA_EINVAL, "spectrum window longer than 1e6 steps: raise nf_min");
                Mv[k] = (int)Mk;
                Mh = std::max(Mh, Mv[k]);
                sc[k] = f * (2.0 / Mk) * (2.0 / Mk) * d.dx * d.dy / (2.0 * kMu0);
            }
            spec_omega = (double*)mem.get((size_t)nf * 8);
            spec_M = (int*)mem.get((size_t)nf * 4);
            spec_scale = (double*)mem.get((size_t)nf * 8);
            spec_ring = (double*)mem.get((size_t)Mh * 4 * plane * 8);
            spec_acc = (double*)mem.get((size_t)nf * 8 * plane * 8);
            spec_partial = (double*)mem.get((size_t)nf * npartial * 8);
            if (!spec_omega || !spec_M || !spec_scale || !spec_ring || !spec_acc || !spec_partial)
                return fail(MITHRA_ENOMEM, "device allocation failed (spectrum)");
            CU(cudaMemcpyAsync(spec_omega, om.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, stream));
            CU(cudaMemcpyAsync(spec_M, Mv.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, stream));
            CU(cudaMemcpyAsync(spec_scale, sc.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, stream));
            CU(cudaMemsetAsync(spec_ring, 0, (size_t)Mh * 4 * plane * 8, stream));
            CU(cudaMemsetAsync(spec_acc, 0, (size_t)nf * 8 * plane * 8, stream));
            CU(cudaStreamSynchronize(stream));   // the host vectors go out of scope
        }
        if (bunch_every > 0 && !(bunch_partial = (double*)mem.get((size_t)14 * npartial * 8)))
            return fail(MITHRA_ENOMEM, "device allocation failed (bunch sampling)");
        for (int b = 0; b < 2; ++b)
            if (!(box[b] = (int*)mem.get((size_t)deposit_box_words(g.nz) * sizeof(int))))
                return fail(MITHRA_ENOMEM, "device allocation failed (box)");
        if (!(box_rec = (int*)mem.get((size_t)6 * std::max<int64_t>(push_blocks(np), 1) * sizeof(int))))
            return fail(MITHRA_ENOMEM, "device allocation failed (box records)");
        if (ef.kind == 0 || ef.kind == 1) {
            for (int b = 0; b < (ef.kind == 1 ? 2 : 1); ++b) {
                if (sizeof(real) == 8) ptab[b] = (double2*)mem.get((size_t)g.nz * sizeof(double2));
                else ptab32[b] = (float4*)mem.get((size_t)g.nz * 2 * sizeof(float4));
                if (!ptab[b] && !ptab32[b]) return fail(MITHRA_ENOMEM, "device allocation failed (phase table)");
            }
        }
        if (ef.kind == 4 && sizeof(real) == 4) {
            // FP32-mixed array: the planar table per module plus the modules' peak fields (the
            // FP64 path evaluates the array directly)
            ptab32[0] = (float4*)mem.get((size_t)g.nz * 2 * sizeof(float4));
            ptab32a = (float4*)mem.get((size_t)g.nz * sizeof(float4));
            if (!ptab32[0] || !ptab32a) return fail(MITHRA_ENOMEM, "device allocation failed (phase table)");
        }
        if (!(err_word = (int*)mem.get(sizeof(int)))) return fail(MITHRA_ENOMEM, "device allocation failed (error word)");
        CU(cudaMemsetAsync(err_word, 0, sizeof(int), stream));
        if (!(counters = (unsigned*)mem.get(2 * sizeof(unsigned))))
            return fail(MITHRA_ENOMEM, "device allocation failed (counters)");
        CU(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned), stream));
        // the state and, in sd[1], the next step's, formed by the step tail's phase-table blocks
        if (!(sd = (StepDev*)mem.get(2 * sizeof(StepDev)))) return fail(MITHRA_ENOMEM, "device allocation failed (step state)");
        CU(cudaMemsetAsync(sd, 0, 2 * sizeof(StepDev), stream));   // the counter starts at step 0
        scst.T0 = d.T0;
        scst.dt = d.dt;
        scst.g0 = d.g0;
        scst.b0 = d.b0;
        scst.z0 = d.z0;
        scst.omega_h = d.omega_h;
        scst.M = (int)d.M;
        CU(launch_step_init(sd, scst, phase_tables(), stream));   // step 0's state and phase tables
        const char* no_graph = std::getenv("MITHRA_NO_GRAPHS");
        use_graphs = !(no_graph && no_graph[0] == '1');
        const char* no_tma = std::getenv("MITHRA_NO_TMA");
        if (!(no_tma && no_tma[0] == '1')) tma = make_tma_maps<real>(pot, src, g);
        // failure tests: MITHRA_TEST_TMA_SKIP_PLANE=p makes every TMA stencil block leave its p-th
        // plane uncopied, so that its bounded wait expires and mithra_sync reports ETIMEDOUT
        const char* skip = std::getenv("MITHRA_TEST_TMA_SKIP_PLANE");
        test_tma_skip = (skip && skip[0] >= '0' && skip[0] <= '9') ? std::atoi(skip) : -1;
        murc = mur_face_coef(g, mur_order);
        int rc = full_box(nstep % 2);
        if (rc) return rc;
        return grow_series(1024);
    }

    int64_t bunch_rows(int64_t steps) const { return bunch_every > 0 ? (steps + bunch_every - 1) / bunch_every : 0; }

    // Grow every per-step series to hold `need` steps (old and new buffers while copying).
    int grow_series(int64_t need)
    {
        if (need <= ser_cap) return MITHRA_OK;
        int64_t cap = ser_cap ? ser_cap : 1024;
        while (cap < need) cap *= 2;
        double* np_ = (double*)mem.get((size_t)cap * 8);
        double* ne_ = (double*)mem.get((size_t)cap * 8);
        double* ns_ = nf > 0 ? (double*)mem.get((size_t)cap * nf * 8) : nullptr;
        double* nb_ = bunch_every > 0 ? (double*)mem.get((size_t)bunch_rows(cap) * 15 * 8) : nullptr;
        if (!np_ || !ne_ || (nf > 0 && !ns_) || (bunch_every > 0 && !nb_))
            return fail(MITHRA_ENOMEM, "device allocation failed (series)");
        CU(cudaMemsetAsync(np_, 0, (size_t)cap * 8, stream));
        CU(cudaMemsetAsync(ne_, 0, (size_t)cap * 8, stream));
        if (ns_) CU(cudaMemsetAsync(ns_, 0, (size_t)cap * nf * 8, stream));
        if (nb_) CU(cudaMemsetAsync(nb_, 0, (size_t)bunch_rows(cap) * 15 * 8, stream));
        graph_reset();   // the captured steps write into the old series
        if (ser_cap) {
            CU(cudaMemcpyAsync(np_, ser_p, (size_t)ser_cap * 8, cudaMemcpyDeviceToDevice, stream));
            CU(cudaMemcpyAsync(ne_, ser_e, (size_t)ser_cap * 8, cudaMemcpyDeviceToDevice, stream));
            if (ns_) CU(cudaMemcpyAsync(ns_, ser_s, (size_t)ser_cap * nf * 8, cudaMemcpyDeviceToDevice, stream));
            if (nb_)
                CU(cudaMemcpyAsync(nb_, ser_b, (size_t)bunch_rows(ser_cap) * 15 * 8, cudaMemcpyDeviceToDevice, stream));
            CU(cudaStreamSynchronize(stream));
            mem.release(ser_p);
            mem.release(ser_e);
            if (ser_s) mem.release(ser_s);
            if (ser_b) mem.release(ser_b);
        }
        ser_p = np_;
        ser_e = ne_;
        ser_s = ns_;
        ser_b = nb_;
        ser_cap = cap;
        return MITHRA_OK;
    }

    void pbeg(int kid, cudaEvent_t* a)
    {
        if (!prof) return;
        *a = ev_get();
        cudaEventRecord(*a, stream);
        (void)kid;
    }
    void pend(int kid, cudaEvent_t a)
    {
        if (!prof) return;
        cudaEvent_t b = ev_get();
        cudaEventRecord(b, stream);
        prof_pending.push_back({kid, a, b});
    }

    // The phase tables the push reads (filled for step n + 1 by step n's tail).
    PhaseTables phase_tables() const
    {
        PhaseTables pt;
        pt.ef = ef;
        pt.kz = d.g0 * d.dz;
        pt.nz = g.nz;
        pt.t32[0] = ptab32[0];
        pt.t32[1] = ptab32[1];
        pt.ta32 = ptab32a;
        pt.t64[0] = ptab[0];
        pt.t64[1] = ptab[1];
        return pt;
    }

    FieldLevels<real> levels() const
    {
        FieldLevels<real> L;
        for (int c = 0; c < 4; ++c) {
            L.n0[c] = pot[lev(0)][c];
            L.n1[c] = pot[lev(1)][c];
            L.out[c] = pot[lev(2)][c];
            L.src[c] = src[c];
        }
        return L;
    }

    int sort_now()
    {
        cudaEvent_t e0 = nullptr;
        pbeg(MITHRA_K_SORT, &e0);
        CU(launch_sort<real>(P, T, np, g, ss, stream));
        pend(MITHRA_K_SORT, e0);
        return MITHRA_OK;
    }

    // One field step (launches only).  Host state advanced here: the level ring, the step count
    // and, on sort steps, the particle buffers.
    int one_step()
    {
        const int ncomp = g.space_charge ? 4 : 3;
        Fields6<real> E6;
        E6.p = eb;
        Fields4<real> S4;
        for (int c = 0; c < 4; ++c) S4.c[c] = src[c];
        int rc = MITHRA_OK;
        const int64_t n = nstep;
        if (sort_every > 0 && n > 0 && n % sort_every == 0 && np > 1) {
            if ((rc = sort_now())) return rc;
        }
        FieldLevels<real> L = levels();
        cudaEvent_t e0 = nullptr;
        // E/B where the particles are (and on the power plane); clears the previous sources
        EmitBox bx{box[n % 2], box[(n + 1) % 2], (int)d.kp, true};
        EmitMaps em;
        if (emit_maps(tma, lev(0), lev(1), &em)) bx.maps = &em;
        bx.err = err_word;
        pbeg(MITHRA_K_EMIT, &e0);
        CU(launch_emit<real>(L, E6, g, bx, stream));
        pend(MITHRA_K_EMIT, e0);
        PushConst pc;
        pc.sd = sd;
        pc.qJ[0] = d.q / (d.dy * d.dz * d.dt);
        pc.qJ[1] = d.q / (d.dz * d.dx * d.dt);
        pc.qJ[2] = d.q / (d.dx * d.dy * d.dt);
        pc.qrho = d.q / (d.dx * d.dy * d.dz);
        pc.cdtb[0] = kC * d.dtb / d.dx;
        pc.cdtb[1] = kC * d.dtb / d.dy;
        pc.cdtb[2] = kC * d.dtb / d.dz;
        pc.ptab[0] = ptab[0];
        pc.ptab[1] = ptab[1];
        pc.ptab32[0] = ptab32[0];
        pc.ptab32[1] = ptab32[1];
        pc.ptab32a = ptab32a;
        pc.kugf = (float)(ef.ku * ef.gap);
        pc.pwinf = ef.gap > 0.0 ? (float)(kPi / (ef.ku * ef.gap)) : 0.f;
        pc.egbf = (float)(ef.g0 * ef.b0 * kC);
        pc.gbf = (float)ef.g0;
        pc.kz = d.g0 * d.dz;
        pc.zstep = d.g0 * d.b0 * kC * d.dtb;
        pc.kdz = (float)(ef.ku * pc.kz);
        pc.kzs = (float)(ef.ku * pc.zstep);
        pc.x0f = (float)g.x0;
        pc.y0f = (float)g.y0;
        pc.dxf = (float)g.dx;
        pc.dyf = (float)g.dy;
        pc.dtbf = (float)g.dtb;
        pc.qrhof = (float)pc.qrho;
        pc.kuf = (float)ef.ku;
        pc.cpolf = (float)ef.cpol;
        pc.spolf = (float)ef.spol;
        for (int l = 0; l < 3; ++l) {
            pc.qJf[l] = (float)pc.qJ[l];
            pc.cdtbf[l] = (float)pc.cdtb[l];
        }
        for (int l = 0; l < 4; ++l) {
            const double qa = fabs(l < 3 ? pc.qJ[l] : pc.qrho);
            const double sc = qa > 0.0 ? 1073741824.0 / (128.0 * qa) : 1.0;
            pc.tscale[l] = (float)sc;
            pc.tunit[l] = (float)(1.0 / (double)pc.tscale[l]);
            (l < 3 ? pc.qJt[l] : pc.qrhot) = (float)((l < 3 ? pc.qJ[l] : pc.qrho) * (double)pc.tscale[l]);
        }
        pc.eB0f = (float)(ef.g0 * ef.b0 * kC * ef.B0);
        pc.bB0f = (float)(ef.g0 * ef.B0);
        pc.B0f = (float)ef.B0;
        pc.ltE = (float)(ef.g0 * (1.0 + ef.b0) * ef.E0);
        pc.ltB = (float)(ef.g0 * (1.0 + ef.b0) * ef.E0 / kC);
        pc.E0f = (float)ef.E0;
        pc.E0cf = (float)(ef.E0 / kC);
        pc.w0f = (float)ef.w0;
        pc.izrf = (float)(1.0 / ef.zr);
        pc.zrf = (float)ef.zr;
        pc.kLf = (float)ef.kL;
        int* far = box[(n + 1) % 2] + deposit_box_ints(g.nz);   // reset by this step's emission
        pc.far = far;
        pbeg(MITHRA_K_PUSH, &e0);
        CU(launch_push<real>(P, np, g, ef, E6, S4, pc, box_rec, stream));
        pend(MITHRA_K_PUSH, e0);
        if (bunch_every > 0) {
            pbeg(MITHRA_K_POWER, &e0);
            BunchSample bs;
            bs.sd = sd;
            bs.every = bunch_every;
            bs.shift[0] = g.x0 + 0.5 * (g.nx - 1) * g.dx;
            bs.shift[1] = g.y0 + 0.5 * (g.ny - 1) * g.dy;
            bs.shift[2] = g.z0 + 0.5 * (g.nz - 1) * g.dz;
            bs.shift[3] = bs.shift[4] = bs.shift[5] = 0.0;
            bs.shift[6] = bunch_shift_g;
            bs.g0 = d.g0;
            bs.b0 = d.b0;
            bs.T0 = d.T0;
            bs.dt = d.dt;
            CU(launch_bunch_sample<real>(P, np, g, bs, bunch_partial, npartial, ser_b, stream));
            pend(MITHRA_K_POWER, e0);
        }
        pbeg(MITHRA_K_STENCIL, &e0);
        if (tma) {
            real* outp[4] = {pot[lev(2)][0], pot[lev(2)][1], pot[lev(2)][2], pot[lev(2)][3]};
            real* prevp[4] = {pot[lev(0)][0], pot[lev(0)][1], pot[lev(0)][2], pot[lev(0)][3]};
            // the sources lie in the nodes of the last deposit box grown by one cell per sub-step,
            // unless the push set the far flag
            CU(launch_stencil_tma<real>(tma, outp, prevp, &murc, lev(1), lev(0), g, cf, ncomp, box[n % 2], far,
                                        g.substeps, err_word, stream, test_tma_skip));
        } else {
            CU(launch_stencil<real>(L, g, cf, ncomp, stream));
        }
        const bool xf = tma != nullptr && tma_x_faces<real>();   // the stencil wrote the Mur x faces
        if (seed.type >= 0) {
            real* outs[2] = {pot[lev(2)][0], pot[lev(2)][1]};
            CU(launch_tfsf<real>(outs, g, cf, seed, sd, d.T0, seed_buf, stream));
            // the x-face nodes next to the corrected planes see their new inward neighbours
            if (xf) CU(launch_mur_tfsf_xfaces<real>(L, g, mur_order, stream));
        }
        pend(MITHRA_K_STENCIL, e0);
        if (nf > 0) {
            // the spectrum reads this step's state: before the tail advances it
            pbeg(MITHRA_K_POWER, &e0);
            SpecStep sp;
            sp.kp = (int)d.kp;
            sp.nf = nf;
            sp.Mh = Mh;
            sp.sd = sd;
            sp.dt = d.dt;
            sp.omega = spec_omega;
            sp.M = spec_M;
            sp.scale = spec_scale;
            sp.ring = spec_ring;
            sp.acc = spec_acc;
            CU(launch_spectrum_step<real>(E6, g, sp, spec_partial, npartial, ser_s, stream));
            pend(MITHRA_K_POWER, e0);
        }
        // Mur faces, then the step tail: the edges and corners, the radiated power of the step,
        // the phase tables of the next step and the step state's advance
        pbeg(MITHRA_K_MUR, &e0);
        {
            if (!ring || !acc || !partial) return fail(MITHRA_EINVAL, "power diagnostic buffers missing");
            const int M = (int)d.M;
            StepTail tl;
            tl.eb = eb;
            tl.power.kp = (int)d.kp;
            tl.power.ring = ring;
            tl.power.acc = acc;
            tl.power.onaxis_id = onaxis_id;
            tl.power.onaxis_series = ser_e;
            const double f = d.g0 * d.g0 * (1.0 + d.b0) * (1.0 + d.b0);
            tl.power.scale = f * (2.0 / M) * (2.0 / M) * d.dx * d.dy / (2.0 * kMu0);
            tl.power.series = ser_p;
            tl.partial = partial;
            tl.npartial = npartial;
            tl.phase = phase_tables();
            tl.sd = sd;
            tl.sc = scst;
            tl.box_rec = box_rec;
            tl.nrec = np > 0 ? push_blocks(np) : 0;
            tl.box_out = box[(n + 1) % 2];   // reset by this step's emission
            CU(launch_mur<real>(L, g, mur_order, ncomp, xf, counters, tl, stream));
        }
        pend(MITHRA_K_MUR, e0);
        base = (base + 1) % 3;
        ++nstep;
        if (prof && prof_pending.size() > 4096) {
            CU(cudaStreamSynchronize(stream));
            prof_collect();
        }
        return rc;
    }

    // Steps per captured graph: the level ring (3), the deposit boxes (2) and the particle
    // buffers swapped by every sort (2 sort periods) all return to their state after it; 0 when
    // that period is too long to capture.
    int64_t graph_period() const
    {
        int64_t L = 6;
        if (sort_every > 0 && np > 1) {
            const int64_t s2 = 2 * (int64_t)sort_every;
            int64_t a = L, b = s2;
            while (b) {
                const int64_t t = a % b;
                a = b;
                b = t;
            }
            L = L / a * s2;
        }
        return L <= kGraphMaxSteps ? L : 0;
    }

    void graph_reset()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gtmpl) cudaGraphDestroy(gtmpl);
        gexec = nullptr;
        gtmpl = nullptr;
        glen = 0;
        gnodes = 0;
    }

    // The captured period as a graph, when the next steps are exactly one replay of it: at an
    // aligned step with at least a period left, and with room in the series for it (growing the
    // series re-captures).  The caller launches it (inside a graph of its own) and then calls
    // period_replayed().
    cudaGraph_t period_graph(int64_t steps_left) override
    {
        const int64_t L = graph_steps();
        if (L <= 0 || !gexec || !gtmpl || glen != L || nstep < L || nstep % L != 0 || steps_left < L) return nullptr;
        if (grow_series(nstep + L) != MITHRA_OK) return nullptr;
        return gexec ? gtmpl : nullptr;
    }
    void period_replayed() override
    {
        nstep += glen;
        count_launches(gnodes);
    }

    // Capture the L steps from an aligned step (a multiple of L, after the first period) into a
    // graph and run it.  The capture advances the host state by L steps, exactly as running them
    // does; the graph then does the device work.
    int graph_capture_run(int64_t L)
    {
        const int base0 = base;
        const Particles<real> P0 = P;
        const int64_t l0 = launch_count();
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(MITHRA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        int rc = MITHRA_OK;
        for (int64_t k = 0; k < L && rc == MITHRA_OK; ++k) rc = one_step();
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(stream, &gr);
        if (rc != MITHRA_OK || e != cudaSuccess || !gr) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            return rc != MITHRA_OK ? rc : fail(MITHRA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        if (base != base0 || P.ix != P0.ix) {
            cudaGraphDestroy(gr);
            return fail(MITHRA_ECUDA, "graph capture: the step state is not periodic");
        }
        e = cudaGraphInstantiate(&gexec, gr, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(gr);
            gexec = nullptr;
            return fail(MITHRA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        gtmpl = gr;
        glen = L;
        gnodes = launch_count() - l0;
        CU(cudaGraphLaunch(gexec, stream));
        return MITHRA_OK;
    }

    int64_t graph_steps() const override { return (use_graphs && !prof && stream) ? graph_period() : 0; }

    int step(int64_t nsteps) override
    {
        int rc = grow_series(nstep + nsteps);
        if (rc) return rc;
        int64_t s = 0;
        while (s < nsteps) {
            // capture needs a created stream (not the legacy default one)
            const int64_t L = graph_steps();
            if (L > 0 && nstep >= L && nstep % L == 0 && nsteps - s >= L) {
                if (gexec && glen == L) {
                    CU(cudaGraphLaunch(gexec, stream));
                    count_launches(gnodes);
                    nstep += L;
                } else {
                    graph_reset();
                    if ((rc = graph_capture_run(L))) return rc;
                }
                s += L;
                continue;
            }
            if ((rc = one_step())) return rc;
            ++s;
        }
        return MITHRA_OK;
    }

    real* field_ptr(int which, int level)
    {
        if (which < 4) return pot[lev(level)][which];
        if (which < 8) return src[which - 4];
        return eb;   // interleaved: component which - 8 of every kEBStride values
    }

    int fields(int which, int level, double* out, size_t cap) override
    {
        if (which < 0 || which > 13 || level < 0 || level > 1) return fail(MITHRA_EINVAL, "fields: bad index/level");
        if (cap < (size_t)g.ncell) return fail(MITHRA_ERANGE, "fields: buffer too small");
        if (which >= 8) {
            const int rc = emit_full();
            if (rc) return rc;
        }
        if (which >= 8) {
            // E, B: a strided device-to-host copy of one component of the interleaved array
            std::vector<real> h((size_t)g.ncell);
            CU(cudaMemcpy2DAsync(h.data(), sizeof(real), eb + (which - 8), kEBStride * sizeof(real), sizeof(real),
                                 (size_t)g.ncell, cudaMemcpyDeviceToHost, stream));
            CU(cudaStreamSynchronize(stream));
            for (int64_t i = 0; i < g.ncell; ++i) out[i] = (double)h[(size_t)i];
            return MITHRA_OK;
        }
        std::vector<real> h((size_t)g.ncell);
        CU(cudaMemcpyAsync(h.data(), field_ptr(which, level), (size_t)g.ncell * sizeof(real), cudaMemcpyDeviceToHost,
                           stream));
        CU(cudaStreamSynchronize(stream));
        for (int64_t i = 0; i < g.ncell; ++i) out[i] = (double)h[(size_t)i];
        return MITHRA_OK;
    }

    int set_field(int which, int level, const double* in, size_t n) override
    {
        if (which < 0 || which > 3 || level < 0 || level > 1) return fail(MITHRA_EINVAL, "set_field: bad index/level");
        if (n != (size_t)g.ncell) return fail(MITHRA_EINVAL, "set_field: size must be nx*ny*nz");
        std::vector<real> h((size_t)g.ncell);
        for (int64_t i = 0; i < g.ncell; ++i) h[(size_t)i] = (real)in[i];
        CU(cudaMemcpyAsync(field_ptr(which, level), h.data(), (size_t)g.ncell * sizeof(real), cudaMemcpyHostToDevice,
                           stream));
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    int ensure_rest_buf()
    {
        if (!rest_buf) rest_buf = (double*)mem.get((size_t)(np > 0 ? np : 1) * 6 * 8);
        return rest_buf ? MITHRA_OK : fail(MITHRA_ENOMEM, "device allocation failed (particle staging)");
    }

    int particles(double* out, size_t cap) override
    {
        if (cap < (size_t)np) return fail(MITHRA_ERANGE, "particles: buffer too small");
        if (np == 0) return MITHRA_OK;
        int rc = ensure_rest_buf();
        if (rc) return rc;
        CU(launch_get_rest<real>(P, np, g, rest_buf, stream));
        CU(cudaMemcpyAsync(out, rest_buf, (size_t)np * 6 * 8, cudaMemcpyDeviceToHost, stream));
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    int set_particles(const double* in, size_t n) override
    {
        if (n != (size_t)np) return fail(MITHRA_EINVAL, "set_particles: row count must equal the bunch size");
        if (np == 0) return MITHRA_OK;
        int rc = ensure_rest_buf();
        if (rc) return rc;
        CU(cudaMemcpyAsync(rest_buf, in, (size_t)np * 6 * 8, cudaMemcpyHostToDevice, stream));
        CU(launch_set_rest<real>(rest_buf, np, P, g, stream));
        CU(cudaStreamSynchronize(stream));
        return full_box(nstep % 2);
    }

    int diag(double* fe, double* b3) override
    {
        Fields6<real> E6;
        E6.p = eb;
        double h[4] = {0, 0, 0, 0};
        if (fe) {
            const int rc = emit_full();
            if (rc) return rc;
            CU(launch_energy<real>(E6, g, partial, npartial, small, stream));
        }
        if (b3) CU(launch_bunching<real>(P, np, g, d.kb, partial + npartial, npartial, small + 4, btab, stream));
        CU(cudaMemcpyAsync(h, small, 8, cudaMemcpyDeviceToHost, stream));
        double hb[3] = {0, 0, 0};
        CU(cudaMemcpyAsync(hb, small + 4, 24, cudaMemcpyDeviceToHost, stream));
        CU(cudaStreamSynchronize(stream));
        if (fe) *fe = h[0];
        if (b3) {
            b3[0] = hb[0];
            b3[1] = hb[1];
            b3[2] = hb[2];
        }
        if (fe && !std::isfinite(h[0])) return fail(MITHRA_EDIVERGED, "field energy is not finite");
        return MITHRA_OK;
    }

    int series(int which, double* out, size_t cap, size_t* n_out) override
    {
        if (n_out) *n_out = (size_t)nstep;
        if (!out) return MITHRA_OK;
        if (cap < (size_t)nstep) return fail(MITHRA_ERANGE, "series: buffer too small");
        if (nstep == 0) return MITHRA_OK;
        if (which == 0) {
            CU(cudaMemcpyAsync(out, ser_p, (size_t)nstep * 8, cudaMemcpyDeviceToHost, stream));
        } else {
            CU(cudaMemcpyAsync(out, ser_e, (size_t)nstep * 8, cudaMemcpyDeviceToHost, stream));
        }
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    int set_seed(const mithra_seed& in) override
    {
        if (nstep > 0) return fail(MITHRA_EINVAL, "set_seed: the run has already stepped");
        if (in.type < -1 || in.type > 1) return fail(MITHRA_EINVAL, "set_seed: unknown seed type");
        for (double v : {in.a0, in.lambda, in.pol_deg, in.waist, in.focus, in.offset, in.pulse_fwhm, in.cep_deg})
            if (!std::isfinite(v)) return fail(MITHRA_EINVAL, "set_seed: non-finite value");
        if (in.type >= 0 && !(in.lambda > 0.0)) return fail(MITHRA_EINVAL, "set_seed: lambda must be > 0");
        if (in.type == 1 && !(in.waist > 0.0)) return fail(MITHRA_EINVAL, "set_seed: waist must be > 0");
        graph_reset();   // the captured steps do not hold the TF/SF kernels
        SeedField s{};
        s.type = in.type;
        if (in.type >= 0) {
            s.g0 = d.g0;
            s.b0 = d.b0;
            s.A0 = in.a0 * kMe * kC / kQe;
            s.k = 2.0 * kPi / in.lambda;
            s.w = kC * s.k;
            s.w0 = in.type == 1 ? in.waist : 0.0;
            s.zr = in.type == 1 ? kPi * in.waist * in.waist / in.lambda : 1.0;
            s.focus = in.focus;
            s.t0 = in.offset / kC;
            s.tp = in.pulse_fwhm / kC;
            s.cep = in.cep_deg * kPi / 180.0;
            s.cpol = std::cos(in.pol_deg * kPi / 180.0);
            s.spol = std::sin(in.pol_deg * kPi / 180.0);
            if (!seed_buf && !(seed_buf = (double*)mem.get((size_t)4 * g.nx * g.ny * 8)))
                return fail(MITHRA_ENOMEM, "device allocation failed (seed planes)");
        }
        seed = s;
        return MITHRA_OK;
    }

    int spectrum(double* h, double* p, size_t cap, size_t* n_steps) override
    {
        if (nf <= 0) return fail(MITHRA_EINVAL, "spectrum: the run has no frequency sweep (nf_points = 0)");
        if (n_steps) *n_steps = (size_t)nstep;
        if (h) std::memcpy(h, hk.data(), (size_t)nf * sizeof(double));
        if (!p || nstep == 0) return MITHRA_OK;
        if (cap < (size_t)nstep * (size_t)nf) return fail(MITHRA_ERANGE, "spectrum: buffer too small");
        CU(cudaMemcpyAsync(p, ser_s, (size_t)nstep * nf * 8, cudaMemcpyDeviceToHost, stream));
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    int bunch_samples(double* out, size_t cap_rows, size_t* n_rows) override
    {
        if (bunch_every <= 0) return fail(MITHRA_EINVAL, "bunch_series: bunch sampling is off (bunch_every = 0)");
        const int64_t rows = bunch_rows(nstep);
        if (n_rows) *n_rows = (size_t)rows;
        if (!out || rows == 0) return MITHRA_OK;
        if (cap_rows < (size_t)rows) return fail(MITHRA_ERANGE, "bunch_series: buffer too small");
        CU(cudaMemcpyAsync(out, ser_b, (size_t)rows * 15 * 8, cudaMemcpyDeviceToHost, stream));
        CU(cudaStreamSynchronize(stream));
        return MITHRA_OK;
    }

    int sync() override
    {
        CU(cudaStreamSynchronize(stream));
        if (prof) prof_collect();
        int e = 0;
        CU(cudaMemcpy(&e, err_word, sizeof e, cudaMemcpyDeviceToHost));
        if (e) return fail(MITHRA_ETIMEDOUT, "a bounded device-side wait expired (TMA copy never completed)");
        return MITHRA_OK;
    }

    void destroy_all() override
    {
        if (stream) cudaStreamSynchronize(stream);
        graph_reset();
        prof_collect();
        free_tma_maps(tma);
        tma = nullptr;
        for (auto e : ev_free) cudaEventDestroy(e);
        ev_free.clear();
        mem.release_all();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
};

bool finite_all(std::initializer_list<double> v)
{
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Rest frame, mesh checks and placement (manual Sec. "Lorentz Transformation", Sec. MESH).
int derive(const mithra_grid& gr, double dt_lab, const mithra_undulator& u, const mithra_bunch& b, Derived& d,
           ExtField& ef)
{
    const int kind = u.kind;
    double g0 = b.gamma;
    // planar (an array's rest frame follows its first module) or linearly polarised laser
    if (kind == 0 || kind == 2 || kind == 3 || kind == 4) g0 = b.gamma / std::sqrt(1.0 + 0.5 * u.K * u.K);
    else if (kind == 1) g0 = b.gamma / std::sqrt(1.0 + u.K * u.K);
    if (!(g0 >= 1.0)) return fail(MITHRA_EINVAL, "gamma0 < 1: raise gamma or lower K");
    d.g0 = g0;
    d.b0 = std::sqrt(1.0 - 1.0 / (g0 * g0));
    d.dz = g0 * gr.dz;
    d.dx = gr.dx;
    d.dy = gr.dy;
    if (gr.solver == 0) {
        const double r2 = (d.dz / d.dx) * (d.dz / d.dx) + (d.dz / d.dy) * (d.dz / d.dy);
        const double ratio = std::sqrt(r2);
        if (ratio >= 1.0) {
            const double s = ratio / 0.99;
            d.dx *= s;
            d.dy *= s;
        }
        const double q2 = (d.dz / d.dx) * (d.dz / d.dx) + (d.dz / d.dy) * (d.dz / d.dy);
        d.A = 0.25 * (1.0 + 0.02 / q2);
        d.dt = d.dz / kC;
    } else {
        d.A = 0.0;
        if (dt_lab > 0.0) {
            d.dt = dt_lab / g0;
        } else {
            if (!(gr.courant > 0.0 && gr.courant < 1.0)) return fail(MITHRA_EINVAL, "FD needs 0 < courant < 1");
            d.dt = gr.courant / (kC * std::sqrt(1.0 / (d.dx * d.dx) + 1.0 / (d.dy * d.dy) + 1.0 / (d.dz * d.dz)));
        }
    }
    const int N = gr.substeps > 0 ? gr.substeps : 1;
    d.dtb = d.dt / N;

    ef = ExtField{};
    ef.kind = kind;
    ef.g0 = d.g0;
    ef.b0 = d.b0;
    const double th = u.pol_deg * kPi / 180.0;
    ef.cpol = std::cos(th);
    ef.spol = std::sin(th);
    const double lam = u.lambda;
    const double kk = 2.0 * kPi / lam;
    ef.ku = kk;
    ef.Lu = u.n_periods * lam;
    ef.B0 = 2.0 * kPi * kMe * kC * u.K / (kQe * lam);
    ef.qlam = 0.25 * lam;
    ef.kL = kk;
    ef.wL = kC * kk;
    ef.E0 = u.K * kMe * kC * ef.wL / kQe;
    ef.tp = u.pulse_fwhm / kC;
    ef.signal = u.signal;
    ef.w0 = (kind == 3) ? u.waist : 0.0;
    ef.zr = (ef.w0 > 0.0) ? kPi * ef.w0 * ef.w0 / lam : 1.0;
    ef.gap = kind == 4 ? u.gap : 0.0;
    ef.nmod = kind == 4 ? u.n_modules : 1;
    ef.dB0 = kind == 4 ? 2.0 * kPi * kMe * kC * u.taper / (kQe * lam) : 0.0;
    const bool stat = kind == 0 || kind == 1 || kind == 4;
    if (stat) d.kstar = d.g0 * d.b0 * kk;
    else if (kind == 2 || kind == 3) d.kstar = d.g0 * (1.0 + d.b0) * kk;
    else d.kstar = kk;
    if (stat) d.kb = d.g0 * kk + d.kstar;
    else if (kind == 2 || kind == 3) d.kb = 2.0 * d.kstar;
    else d.kb = d.kstar;
    d.omega_h = gr.norm_freq * kC * d.kstar;

    // placement: rest coordinates are the boost of lab coordinates measured from the event
    // (t' = 0, undulator entrance).  Static undulator: the run starts when the entrance is
    // dist/gamma0 ahead of the head (head = reference + 3 sig_z), so the lab reference sits at
    // -(dist + gamma0^2 * 3 sig_z) at t' = 0.  Optical: reference at the origin; the pulse centre
    // starts dist ahead and meets the reference at the focus.
    double zeta_ref = 0.0;
    if (stat) zeta_ref = -(u.dist_to_bunch_head + d.g0 * d.g0 * 3.0 * b.sig_z);
    d.z_ref = d.g0 * zeta_ref;
    d.T0 = -d.g0 * d.b0 * zeta_ref / kC;
    ef.t_f = u.dist_to_bunch_head / (kC * (1.0 + d.b0));
    ef.zeta_f = d.b0 * u.dist_to_bunch_head / (1.0 + d.b0);

    d.x0 = gr.cx - 0.5 * (gr.nx - 1) * d.dx;
    d.y0 = gr.cy - 0.5 * (gr.ny - 1) * d.dy;
    d.z0 = d.z_ref + d.g0 * gr.cz - 0.5 * (gr.nz - 1) * d.dz;

    // optimize-bunch-position (Sec. MESH): before the undulator entrance reaches it, the bunch
    // reference (on axis, Lorentz factor gamma) drifts in the rest frame with the relative
    // velocity v = (beta - beta0) / (1 - beta beta0); the entrance, -zeta_ref / gamma0 ahead of it
    // at its time T0, closes in with -beta0 c.  The mesh and the power plane move by the drift
    // v c t up to the meeting, t = (-zeta_ref / gamma0) / ((v + beta0) c), so that the bunch
    // sits at its placed position once it is inside the undulator.
    double shift = 0.0;
    if (gr.optimize_position && stat) {
        const double beta = std::sqrt(1.0 - 1.0 / (b.gamma * b.gamma));
        const double v = (beta - d.b0) / (1.0 - beta * d.b0);
        const double t = (-zeta_ref / d.g0) / ((v + d.b0) * kC);
        shift = v * kC * t;
    }
    d.z0 += shift;

    const double zp = d.z_ref + shift + d.g0 * gr.power_plane_dist;
    double kp = std::round((zp - d.z0) / d.dz);
    if (kp < 1) kp = 1;
    if (kp > gr.nz - 2) kp = gr.nz - 2;
    d.kp = kp;
    double M = std::round(2.0 * kPi / (d.omega_h * d.dt));
    if (!(M >= 1.0)) M = 1.0;
    if (M > 1e6) return fail(MITHRA_EINVAL, "power window longer than 1e6 steps: check norm_freq / lambda");
    d.M = M;
    d.q = b.n > 0 ? -kQe * b.charge_e / (double)b.n : 0.0;
    return MITHRA_OK;
}

template <typename real>
int create_t(const mithra_grid& gr, double dt_lab, const mithra_undulator& u, const mithra_bunch& b,
             const Allocator& alloc, mithra_t* out)
{
    RunT<real>* r = new RunT<real>();
    r->mem.a = alloc;
    int rc = derive(gr, dt_lab, u, b, r->d, r->ef);
    if (rc) {
        delete r;
        return rc;
    }
    const Derived& d = r->d;
    r->precision = gr.precision;
    r->mur_order = gr.mur_order;
    r->sort_every = gr.sort_every == 0 ? 20 : gr.sort_every;
    r->nf = gr.nf_points;
    for (int k = 0; k < r->nf; ++k)
        r->hk.push_back(r->nf == 1 ? gr.nf_min : gr.nf_min + k * (gr.nf_max - gr.nf_min) / (r->nf - 1));
    r->bunch_every = gr.bunch_every;
    r->bunch_shift_g = b.gamma;
    r->np = b.n;
    Geom& g = r->g;
    g.nx = gr.nx;
    g.ny = gr.ny;
    g.nz = gr.nz;
    g.sy = gr.nx;
    g.sz = (int64_t)gr.nx * gr.ny;
    g.ncell = g.sz * gr.nz;
    g.dx = d.dx;
    g.dy = d.dy;
    g.dz = d.dz;
    g.dt = d.dt;
    g.dtb = d.dtb;
    g.x0 = d.x0;
    g.y0 = d.y0;
    g.z0 = d.z0;
    g.substeps = gr.substeps > 0 ? gr.substeps : 1;
    g.space_charge = gr.space_charge ? 1 : 0;
    const double cdt = kC * d.dt;
    const double rx = (cdt / d.dx) * (cdt / d.dx), ry = (cdt / d.dy) * (cdt / d.dy), rz = (cdt / d.dz) * (cdt / d.dz);
    r->cf.a1 = 2.0 * (1.0 - (1.0 - 2.0 * d.A) * rx - (1.0 - 2.0 * d.A) * ry - rz);
    r->cf.ax = rx;
    r->cf.ay = ry;
    r->cf.a6 = rz - 2.0 * d.A * rx - 2.0 * d.A * ry;
    r->cf.w = d.A;
    r->cf.w0 = 1.0 - 2.0 * d.A;
    r->cf.s_a = cdt * cdt * kMu0;
    r->cf.s_phi = cdt * cdt * (kMu0 * kC * kC);   // 1/eps0 = mu0 c^2
    r->onaxis_id = (int64_t)d.kp * g.sz + (int64_t)(gr.ny / 2) * g.sy + gr.nx / 2;

    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete r;
        return fail(MITHRA_ECUDA, "cudaStreamCreateWithFlags failed");
    }
    r->own_stream = true;
    {
        // the run's arrays for its first 1024 steps, without the boost's temporary lab copy
        const int64_t nb = b.n > 0 ? b.n : 1;
        r->mem.reserve((size_t)(mithra::footprint(&gr, &u, &b, 1024) - ((nb * 48 + 255) & ~(int64_t)255)));
    }
    if ((rc = r->alloc_all())) {
        r->destroy_all();
        delete r;
        return rc;
    }
    if (b.n > 0) {
        double* lab = (double*)r->mem.get((size_t)b.n * 6 * 8, true);
        if (!lab) {
            r->destroy_all();
            delete r;
            return fail(MITHRA_ENOMEM, "device allocation failed (lab particles)");
        }
        cudaError_t e = cudaSuccess;
        int* bad = nullptr;   // set on the device when a given particle value is not finite
        if (b.lab_particles) {
            if (!(bad = (int*)r->mem.get(sizeof(int), true))) {
                r->mem.release(lab);
                r->destroy_all();
                delete r;
                return fail(MITHRA_ENOMEM, "device allocation failed (check word)");
            }
            e = cudaMemsetAsync(bad, 0, sizeof(int), r->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(lab, b.lab_particles, (size_t)b.n * 6 * 8, cudaMemcpyHostToDevice, r->stream);
            if (e == cudaSuccess) e = launch_finite_check(lab, (int64_t)b.n * 6, bad, r->stream);
        } else {
            // generated ellipsoid bunch (Sec. BUNCH, bunch-initialization): the quasi-random loader
            // with the bunch's parameters, written straight to device memory
            mithra_ellipsoid el{};
            el.uniform = b.uniform;
            el.gamma = b.gamma;
            el.sig[0] = b.sig_x;
            el.sig[1] = b.sig_y;
            el.sig[2] = b.sig_z;
            el.sig_u[0] = b.sig_x > 0.0 ? b.eps_n_x / b.sig_x : 0.0;
            el.sig_u[1] = b.sig_y > 0.0 ? b.eps_n_y / b.sig_y : 0.0;
            el.sig_u[2] = b.gamma * b.rel_espread;
            el.cse_sigma = b.cse_sigma;
            el.lambda_r = b.lambda_r > 0.0 ? b.lambda_r : 2.0 * kPi / (d.kstar * d.g0 * (1.0 + d.b0));
            el.bunching = b.bunching;
            el.bunching_phase = b.bunching_phase;
            el.shot_noise = b.shot_noise;
            el.charge_e = b.charge_e;
            struct Adapter {
                static void* get(void* c, size_t n) { return ((DevMem*)c)->get(n, true); }
                static void put(void* c, void* q) { ((DevMem*)c)->release(q); }
            };
            rc = ellipsoid_device(el, b.n, b.seed, lab, Adapter::get, Adapter::put, &r->mem, r->stream);
            if (rc) {
                r->mem.release(lab);
                r->destroy_all();
                delete r;
                return rc;
            }
        }
        if (e == cudaSuccess) e = launch_boost<real>(lab, b.n, r->P, g, r->ef, d.z_ref, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        int bad_h = 0;
        if (e == cudaSuccess && bad) e = cudaMemcpy(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost);
        r->mem.release(lab);
        if (bad) r->mem.release(bad);
        if (e != cudaSuccess) {
            r->destroy_all();
            delete r;
            return fail(MITHRA_ECUDA, std::string("particle boost: ") + cudaGetErrorString(e));
        }
        if (bad_h) {
            r->destroy_all();
            delete r;
            return fail(MITHRA_EINVAL, "create: non-finite particle value");
        }
        if (r->sort_every > 0 && b.n > 1 && (rc = r->sort_now())) {
            r->destroy_all();
            delete r;
            return rc;
        }
    }
    cudaError_t e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) {
        r->destroy_all();
        delete r;
        return fail(MITHRA_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = r;
    return MITHRA_OK;
}

}  // namespace

// Checks of mithra_create that need no device (shared with the serving queue).
int mithra::validate_request(const mithra_grid* gr, double dt_lab, const mithra_undulator* u, const mithra_bunch* b)
{
    if (!gr || !u || !b) return fail(MITHRA_EINVAL, "create: null argument");
    if (gr->nx < 6 || gr->ny < 6 || gr->nz < 6) return fail(MITHRA_EINVAL, "create: each axis needs >= 6 nodes");
    if ((int64_t)gr->nx * gr->ny * gr->nz >= (int64_t(1) << 31) - 1)
        return fail(MITHRA_EINVAL, "create: more than 2^31 - 2 nodes");
    if (!finite_all({gr->dx, gr->dy, gr->dz, gr->cx, gr->cy, gr->cz, gr->courant, gr->power_plane_dist, gr->norm_freq,
                     u->K, u->lambda, u->n_periods, u->pol_deg, u->waist, u->pulse_fwhm, u->dist_to_bunch_head, b->gamma,
                     b->charge_e, b->sig_z, dt_lab}))
        return fail(MITHRA_EINVAL, "create: non-finite parameter");
    if (!(gr->dx > 0 && gr->dy > 0 && gr->dz > 0)) return fail(MITHRA_EINVAL, "create: resolution must be > 0");
    if (gr->solver != 0 && gr->solver != 1) return fail(MITHRA_EINVAL, "create: solver must be 0 (NSFD) or 1 (FD)");
    if (gr->mur_order != 1 && gr->mur_order != 2) return fail(MITHRA_EINVAL, "create: mur_order must be 1 or 2");
    if (gr->precision != 0 && gr->precision != 1) return fail(MITHRA_EINVAL, "create: precision must be 0 or 1");
    if (gr->substeps < 0 || gr->substeps > 1024) return fail(MITHRA_EINVAL, "create: substeps out of range");
    if (!(gr->norm_freq > 0)) return fail(MITHRA_EINVAL, "create: norm_freq must be > 0");
    if (gr->nf_points < 0 || gr->nf_points > 256) return fail(MITHRA_EINVAL, "create: nf_points must be 0 .. 256");
    if (gr->nf_points > 0 && !(std::isfinite(gr->nf_min) && std::isfinite(gr->nf_max) && gr->nf_min > 0 &&
                               (gr->nf_points == 1 || gr->nf_max >= gr->nf_min)))
        return fail(MITHRA_EINVAL, "create: spectrum needs 0 < nf_min <= nf_max");
    if (gr->bunch_every < 0) return fail(MITHRA_EINVAL, "create: bunch_every must be >= 0");
    if (gr->optimize_position != 0 && gr->optimize_position != 1)
        return fail(MITHRA_EINVAL, "create: optimize_position must be 0 or 1");
    if (u->kind < -1 || u->kind > 4) return fail(MITHRA_EINVAL, "create: unknown undulator kind");
    if (u->kind == 4) {
        if (!finite_all({u->gap, u->taper}) || !(u->gap >= 0.0))
            return fail(MITHRA_EINVAL, "create: undulator array needs a finite gap >= 0 and a finite taper");
        if (u->n_modules < 1 || u->n_modules > 100000)
            return fail(MITHRA_EINVAL, "create: undulator array needs 1 .. 100000 modules");
        if (!(u->n_periods > 0.0)) return fail(MITHRA_EINVAL, "create: undulator array needs n_periods > 0");
    }
    if (!(u->lambda > 0)) return fail(MITHRA_EINVAL, "create: lambda must be > 0");
    if (!(b->gamma >= 1.0)) return fail(MITHRA_EINVAL, "create: gamma must be >= 1");
    if (b->n < 0 || b->n >= (int64_t(1) << 31)) return fail(MITHRA_EINVAL, "create: particle count out of range");
    if (b->n > 0) {
        if (!(b->charge_e > 0)) return fail(MITHRA_EINVAL, "create: charge_e must be > 0");
        // (non-finite given particle values are found on the device at creation)
        if (!b->lab_particles) {
            if (!finite_all({b->rel_espread, b->sig_x, b->sig_y, b->eps_n_x, b->eps_n_y, b->cse_sigma, b->lambda_r,
                             b->bunching, b->bunching_phase}))
                return fail(MITHRA_EINVAL, "create: non-finite bunch parameter");
            if (!(b->rel_espread >= 0 && b->sig_x >= 0 && b->sig_y >= 0 && b->sig_z >= 0 && b->eps_n_x >= 0 &&
                  b->eps_n_y >= 0 && b->bunching >= 0))
                return fail(MITHRA_EINVAL, "create: bunch sizes, emittances, spread and bunching must be >= 0");
            if ((b->uniform != 0 && b->uniform != 1) || (b->shot_noise != 0 && b->shot_noise != 1))
                return fail(MITHRA_EINVAL, "create: uniform and shot_noise must be 0 or 1");
            if ((uint64_t)b->n + b->seed >= ((uint64_t)1 << 32) - 1)
                return fail(MITHRA_EINVAL, "create: n + seed must be below 2^32 - 1");
        }
    }
    return MITHRA_OK;
}

int mithra::create_with(const mithra_grid* gr, double dt_lab, const mithra_undulator* u, const mithra_bunch* b,
                        mithra_alloc_fn alloc, mithra_free_fn free_fn, void* ctx, mithra_t* out)
{
    if (!out) return fail(MITHRA_EINVAL, "create: null argument");
    *out = nullptr;
    const int rc = validate_request(gr, dt_lab, u, b);
    if (rc) return rc;
    Allocator a;
    a.alloc = alloc;
    a.free_fn = free_fn;
    a.ctx = ctx;
    if (gr->precision == 0) return create_t<double>(*gr, dt_lab, *u, *b, a, out);
    return create_t<float>(*gr, dt_lab, *u, *b, a, out);
}

extern "C" int mithra_create(const mithra_grid* gr, double dt_lab, const mithra_undulator* u, const mithra_bunch* b,
                             mithra_t* out)
{
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    return mithra::create_with(gr, dt_lab, u, b, a.alloc, a.free_fn, a.ctx, out);
}

int64_t mithra::graph_steps(mithra_t r, int64_t* nstep)
{
    if (nstep) *nstep = r ? r->nstep : 0;
    return r ? r->graph_steps() : 0;
}

cudaGraph_t mithra::period_graph(mithra_t r, int64_t steps_left) { return r ? r->period_graph(steps_left) : nullptr; }

void mithra::period_replayed(mithra_t r)
{
    if (r) r->period_replayed();
}

int64_t mithra::footprint(const mithra_grid* gr, const mithra_undulator* u, const mithra_bunch* b, int64_t nsteps)
{
    auto up = [](int64_t x) { return (x + 255) & ~(int64_t)255; };
    const int64_t ncell = (int64_t)gr->nx * gr->ny * gr->nz;
    const int64_t rs = gr->precision == 0 ? 8 : 4;
    const int64_t n = b->n > 0 ? b->n : 1;
    int64_t t = 16 * up(ncell * rs) + up(ncell * rs * kEBStride);             // potentials, sources, E/B
    t += 2 * (4 * up(n * 4) + 3 * up(n * rs) + 3 * up(n * 8));               // particles and sort copy
    t += 2 * up(n * 4) + 2 * up((ncell + 1) * 4) + up((ncell / 4096 + 16) * 4);   // sort scratch
    // the power window M is only known after the rest frame is fixed; bound it by the run's steps
    const int64_t plane = (int64_t)gr->nx * gr->ny;
    const int64_t M = std::min<int64_t>(std::max<int64_t>(nsteps, 1), 4096);
    const int64_t np_ = run_partials(plane);
    t += up(M * 4 * plane * 8) + up(2 * M * 8) + 2 * up(4 * np_ * 8) + up(64);
    int64_t cap = 1024;
    while (cap < nsteps) cap *= 2;
    t += 4 * up(cap * 8);                                                     // series (old and new while growing)
    t += 2 * up(deposit_box_words(gr->nz) * 4) + up(6 * push_blocks(n) * 4) + 2 * up(gr->nz * 32);
    t += up(gr->nz * 16) + up(gr->nz * 8);                                    // phase tables, bunching table
    t += up(n * 48);                                                          // lab particles during the boost
    if (gr->nf_points > 0) {                                                  // spectrum: ring, accumulators, series
        const int64_t nf = gr->nf_points;
        t += up(M * 4 * plane * 8) + up(nf * 8 * plane * 8) + 4 * up(nf * 8) + up(nf * np_ * 8) +
             2 * up(cap * nf * 8);
    }
    if (gr->bunch_every > 0) t += up(14 * np_ * 8) + 2 * up((cap / gr->bunch_every + 1) * 15 * 8);
    // the small buffers (step state, counters, error word, seed planes' bookkeeping) and the 256
    // bytes of alignment slack every allocation takes from a caller's allocator (at most 128)
    t += 128 * 256;
    return t;
}

extern "C" int mithra_set_seed(mithra_t r, const mithra_seed* s)
{
    if (!r || !s) return fail(MITHRA_EINVAL, "set_seed: null argument");
    return r->set_seed(*s);
}

extern "C" int mithra_set_stream(mithra_t r, void* stream)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    CU(cudaStreamSynchronize(r->stream));
    if (r->own_stream) cudaStreamDestroy(r->stream);
    r->own_stream = false;
    r->stream = (cudaStream_t)stream;
    return MITHRA_OK;
}

extern "C" int mithra_step(mithra_t r, int64_t n)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    if (n < 0) return fail(MITHRA_EINVAL, "step: negative count");
    return r->step(n);
}

extern "C" int mithra_sync(mithra_t r)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    return r->sync();
}

extern "C" int mithra_fields(mithra_t r, int which, int level, double* out, size_t cap)
{
    if (!r || !out) return fail(MITHRA_EINVAL, "null argument");
    return r->fields(which, level, out, cap);
}

extern "C" int mithra_set_field(mithra_t r, int which, int level, const double* in, size_t n)
{
    if (!r || !in) return fail(MITHRA_EINVAL, "null argument");
    return r->set_field(which, level, in, n);
}

extern "C" int mithra_particles(mithra_t r, double* out, size_t cap)
{
    if (!r || (!out && r->np > 0)) return fail(MITHRA_EINVAL, "null argument");
    return r->particles(out, cap);
}

extern "C" int mithra_set_particles(mithra_t r, const double* in, size_t n)
{
    if (!r || (!in && n > 0)) return fail(MITHRA_EINVAL, "null argument");
    return r->set_particles(in, n);
}

extern "C" int mithra_radiated_power(mithra_t r, double* p, double* t, size_t cap, size_t* n_out)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    int rc = r->series(0, p, cap, n_out);
    if (rc) return rc;
    if (t) {
        const double zp = r->d.z0 + r->d.kp * r->d.dz;
        for (int64_t i = 0; i < r->nstep; ++i)
            t[i] = r->d.g0 * (r->d.T0 + ((double)i + 0.5) * r->d.dt + r->d.b0 * zp / kC);
    }
    return MITHRA_OK;
}

extern "C" int mithra_power_spectrum(mithra_t r, double* h_out, double* p_lab, size_t cap_values, size_t* n_steps)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    return r->spectrum(h_out, p_lab, cap_values, n_steps);
}

extern "C" int mithra_bunch_series(mithra_t r, double* out15, size_t cap_rows, size_t* n_rows)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    return r->bunch_samples(out15, cap_rows, n_rows);
}

extern "C" int mithra_onaxis_field(mithra_t r, double* ex, size_t cap, size_t* n_out)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    return r->series(1, ex, cap, n_out);
}

extern "C" int mithra_diag(mithra_t r, double* fe, double* b3)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    return r->diag(fe, b3);
}

extern "C" int mithra_info(mithra_t r, double* info, int64_t* hbm)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    if (info) {
        const Derived& d = r->d;
        const double v[19] = {d.g0, d.b0, d.dx, d.dy, d.dz, d.dt, d.dtb, d.A, d.x0, d.y0,
                              d.z0, d.T0, d.omega_h, d.M, d.kp, d.z_ref, d.q, d.kstar, d.kb};
        std::memcpy(info, v, sizeof v);
    }
    if (hbm) *hbm = (int64_t)r->mem.total;
    return MITHRA_OK;
}

extern "C" int mithra_set_profiling(mithra_t r, int on)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    CU(cudaStreamSynchronize(r->stream));
    r->prof_collect();
    for (int k = 0; k < MITHRA_K_COUNT; ++k) {
        r->prof_ms[k] = 0.0;
        r->prof_n[k] = 0;
    }
    r->prof = on != 0;
    return MITHRA_OK;
}

extern "C" int mithra_kernel_stats(mithra_t r, int kid, double* total_ms, int64_t* launches)
{
    if (!r) return fail(MITHRA_EINVAL, "null run");
    if (kid < 0 || kid >= MITHRA_K_COUNT) return fail(MITHRA_EINVAL, "bad kernel id");
    CU(cudaStreamSynchronize(r->stream));
    r->prof_collect();
    if (total_ms) *total_ms = r->prof_ms[kid];
    if (launches) *launches = r->prof_n[kid];
    return MITHRA_OK;
}

extern "C" void mithra_destroy(mithra_t r)
{
    if (!r) return;
    r->destroy_all();
    delete r;
}

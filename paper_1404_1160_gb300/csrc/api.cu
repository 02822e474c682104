// api.cu -- host side of the C ABI declared in include/pic.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pic.h"
#include "pic_internal.h"

using pic::DevParams;

namespace {

constexpr double kPi = 3.14159265358979323846;

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PIC_OK;
    if (e == cudaErrorMemoryAllocation) return PIC_ERR_NO_MEMORY;
    if (e == cudaErrorNotSupported) return PIC_ERR_UNSUPPORTED;
    return PIC_ERR_CUDA;
}

int map_dev(int s) {
    if (s == pic::DEV_OK) return PIC_OK;
    if (s == pic::DEV_TIMEOUT) return PIC_ERR_TIMEOUT;
    return PIC_ERR_CUDA;
}

bool is_pow2(uint64_t w) { return w != 0 && (w & (w - 1)) == 0; }

// Parameter checks shared by every entry point; mesh checks only when the
// Poisson model (or a standalone mesh call) needs the mesh.
int check_params(const pic_params* p, bool need_mesh) {
    if (!p) return PIC_ERR_INVALID_ARG;
    if (!(p->eps > 0.0) || !std::isfinite(p->eps) || !(p->dt > 0.0) || !std::isfinite(p->dt))
        return PIC_ERR_INVALID_ARG;
    if (p->field_model < 0 || p->field_model > 2 || p->fine_solver < 0 || p->fine_solver > 1)
        return PIC_ERR_INVALID_ARG;
    if (p->steps_per_turn < 4 || p->steps_per_turn > (1 << 20)) return PIC_ERR_INVALID_ARG;
    if (p->max_window_steps < 2 * p->steps_per_turn + 2 || p->max_window_steps > (1 << 24))
        return PIC_ERR_INVALID_ARG;
    if (p->precision != 0 && p->precision != 1) return PIC_ERR_INVALID_ARG;
    if (p->precision == 1) {
        // FP32 form: the exact-rotation solver (in the rotating frame), a
        // fixed-point weight that binary32 weights split into 32-bit parts,
        // and dt/h small enough for the compensated time arithmetic
        if (p->fine_solver != PIC_FINE_LAWSON_RK4) return PIC_ERR_UNSUPPORTED;
        if (p->field_model == PIC_FIELD_POISSON && p->weight_fixed > (1ull << 32)) return PIC_ERR_UNSUPPORTED;
        const double D = p->dt / ((2.0 * kPi * p->eps) / (double)p->steps_per_turn);
        if (!(D < 4194304.0)) return PIC_ERR_UNSUPPORTED;
    }
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 1024 || (p->block_size & 31)))
        return PIC_ERR_INVALID_ARG;
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32) return PIC_ERR_INVALID_ARG;
    if (p->sort_every < 0) return PIC_ERR_INVALID_ARG;
    if (p->wait_limit_ns < 0) return PIC_ERR_INVALID_ARG;
    if (p->field_parity != PIC_PARITY_EVEN && p->field_parity != PIC_PARITY_ODD) return PIC_ERR_INVALID_ARG;
    if (need_mesh || p->field_model == PIC_FIELD_POISSON) {
        if (p->n_cells < 2 || p->n_cells > 65536 || (p->n_cells & 1)) return PIC_ERR_INVALID_ARG;
        if (!(p->r_max > 0.0) || !std::isfinite(p->r_max) || p->r_min != -p->r_max) return PIC_ERR_INVALID_ARG;
        if (!is_pow2(p->weight_fixed) || p->weight_fixed > (1ull << 40)) return PIC_ERR_INVALID_ARG;
        if (!(p->total_charge > 0.0) || !std::isfinite(p->total_charge)) return PIC_ERR_INVALID_ARG;
        // fixed-point positions x*W must stay below 2^62
        if ((double)p->n_cells * (double)p->weight_fixed >= 4.611686018427388e18) return PIC_ERR_OVERFLOW;
    }
    return PIC_OK;
}

// Host precomputation of every constant a kernel uses.  The fine step and
// the rotation constants follow h = 2 pi eps / steps_per_turn and
// cos/sin(h/eps), cos/sin(h/(2 eps)) (exact E = 0 flow, Sec. 1).
void make_devparams(const pic_params* p, long long n, DevParams* d) {
    std::memset(d, 0, sizeof(*d));
    d->eps = p->eps;
    d->inv_eps = 1.0 / p->eps;
    d->mie = -d->inv_eps;
    d->h = (2.0 * kPi * p->eps) / (double)p->steps_per_turn;
    d->h2 = 0.5 * d->h;
    d->h6 = d->h / 6.0;
    d->D = p->dt / d->h;
    const double th = d->h / p->eps;
    d->c1 = std::cos(th);
    d->s1 = std::sin(th);
    d->ch = std::cos(0.5 * th);
    d->sh = std::sin(0.5 * th);
    d->hsh = d->h * d->sh;
    d->tch = 2.0 * d->ch;
    d->tsh = 2.0 * d->sh;
    d->n_cells = p->n_cells;
    d->c = p->n_cells / 2;
    d->r_min = p->r_min;
    if (p->n_cells > 0) {
        d->hr = (p->r_max - p->r_min) / (double)p->n_cells;
        d->inv_hr = 1.0 / d->hr;
    }
    d->W = (long long)p->weight_fixed;
    d->Wmask = d->W - 1;
    int l2 = 0;
    while (l2 < 63 && (1ull << l2) < p->weight_fixed) ++l2;
    d->log2W = l2;
    d->Wd = (double)p->weight_fixed;
    d->invW = 1.0 / d->Wd;
    int ex = 0;
    d->xs_fma = (d->inv_hr > 0.0 && std::frexp(d->inv_hr, &ex) == 0.5) ? 1 : 0;
    d->xs_scale = d->inv_hr * d->Wd;
    d->xs_off = -(p->r_min * d->inv_hr) * d->Wd;
    d->xs_max = (double)p->n_cells * d->Wd;
    d->xs_max_i = (long long)p->n_cells * (long long)p->weight_fixed;
    pic::loc_fixed_setup(&d->loc, d->xs_fma, d->xs_scale, d->xs_off, d->xs_max_i, d->log2W);
    d->imul = 1;
    d->q_unit = n > 0 ? p->total_charge / ((double)n * d->Wd) : 0.0;
    d->q_half = 0.5 * d->q_unit;
    d->field = p->field_model;
    d->solver = p->fine_solver;
    d->Kmax = p->max_window_steps;
    d->Tfb = (double)p->steps_per_turn;
    d->n = n;
    d->wait_ns = p->wait_limit_ns > 0 ? p->wait_limit_ns : 2000000000ll;
    d->bar_extra = 0;
    d->parity_odd = p->field_parity == PIC_PARITY_ODD ? 1 : 0;
    // FP32 form: the same constants rounded once to binary32
    d->r_min_f = (float)p->r_min;
    d->inv_hr_f = (float)d->inv_hr;
    d->ncells_f = (float)p->n_cells;
    d->Wf = (float)p->weight_fixed;
    d->h2shh_f = (float)(d->h2 * d->sh);
    d->hshh_f = (float)(d->h * d->sh);
    d->h6_f = (float)d->h6;
    d->spt = p->steps_per_turn;
    const double Dfl = std::floor(d->D);
    d->Di = (int)Dfl;
    d->Df = (float)(d->D - Dfl);
    if (d->Df >= 1.0f) {
        d->Di += 1;
        d->Df = 0.0f;
    }
    d->rot = nullptr;
}

// Fine-step constants for a step of size hstep (the same formulas as
// make_devparams, which uses hstep = 2 pi eps / steps_per_turn).
void set_fine_step(DevParams* d, double eps, double hstep) {
    d->h = hstep;
    d->h2 = 0.5 * hstep;
    d->h6 = hstep / 6.0;
    const double th = hstep / eps;
    d->c1 = std::cos(th);
    d->s1 = std::sin(th);
    d->ch = std::cos(0.5 * th);
    d->sh = std::sin(0.5 * th);
    d->hsh = hstep * d->sh;
    d->tch = 2.0 * d->ch;
    d->tsh = 2.0 * d->sh;
}

// Rotation table of the FP32 form: entry m = (cos, sin)(m pi / spt), the
// exact E = 0 flow over m half fine steps, m = 0 .. 2 spt - 1, in FP64
// rounded once to binary32.  Entries whose exact value is 0 or +-1 (quarter
// turns) are stored exactly.
std::vector<float2> rotation_table(int spt) {
    std::vector<float2> t((size_t)2 * spt);
    for (int m = 0; m < 2 * spt; ++m) {
        float c, sn;
        if ((2 * m) % spt == 0) {  // multiple of a quarter turn
            const int q = (2 * m) / spt;  // 0..3
            const float cq[4] = {1.0f, 0.0f, -1.0f, 0.0f}, sq[4] = {0.0f, 1.0f, 0.0f, -1.0f};
            c = cq[q];
            sn = sq[q];
        } else {
            const double x = kPi * (double)m / (double)spt;
            c = (float)std::cos(x);
            sn = (float)std::sin(x);
        }
        t[(size_t)m] = make_float2(c, sn);
    }
    return t;
}

int current_sm_count(int* sms) {
    int dev = 0, count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return PIC_ERR_CUDA;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return PIC_ERR_CUDA;
    if ((e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return PIC_ERR_CUDA;
    return PIC_OK;
}

cudaMemcpyKind kind_to(int ptr_kind) { return ptr_kind == PIC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_from(int ptr_kind) { return ptr_kind == PIC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

}  // namespace

struct pic_handle {
    pic_params prm;
    DevParams dp;
    long long n = 0;
    cudaStream_t st = nullptr;
    int sm_count = 0, block = 0;
    pic::WinBufs B;
    pic::WindowLaunch L;
    double* Tin = nullptr;   // periods of y^0 (fine steps) when periods_once
    double *tmpR = nullptr, *tmpV = nullptr;  // unpacked R, V for copies in and out
    // storage order: slot s holds original particle perm[s] (phase-space sort)
    int *perm = nullptr, *perm_alt = nullptr;
    double2* y_alt = nullptr;
    double* Tin_alt = nullptr;
    int* skey = nullptr;
    unsigned int* scount = nullptr;
    pic::SortBufs sort;
    std::vector<void*> allocs;
    // field of the current positions
    long long *Qf = nullptr, *nout_f = nullptr;
    double *Ef = nullptr, *edges_f = nullptr;
    void* scan_mem = nullptr;
    pic::ScanScratch S;
    // moments
    double* part_d = nullptr;
    long long* part_i = nullptr;
    int mom_grid = 1;
    int* status_host = nullptr;  // pinned
    // FP32 form (precision 1)
    int prec = 0;
    pic::WinBufs32 B32;
    float2* y32_alt = nullptr;
    pic::CTime *Tin32 = nullptr, *Tin32_alt = nullptr;
    float2* rot32 = nullptr;
    pic::SortBufs32 sort32;
    // learned stepper (allocated by the first pic_step_learned)
    void* y_prev = nullptr;
    double* psi = nullptr;
    float* psi_f = nullptr;    // binary32 field tables of the FP32 form's energy check
    unsigned long long* n_fb = nullptr;
    double t = 0.0;
    long long n_steps = 0;
    int have_periods = 0;
    int band_skip = 0;         // ETD windows left to run with every trajectory row (after a band miss)
    long long band_replays = 0;
    long long launches = 0;
    // CUDA events around the window launches of the last pic_step call
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double window_ms = 0.0;
    int64_t window_n = 0;
    // sums over the windows of one pic_step_classic call
    bool acc_on = false;
    double acc_ms = 0.0;
    int64_t acc_n = 0;
    int64_t acc_fine = 0;
};

namespace {

// Trajectory band of the FP64 ETD window: rows within kBandMargin of the
// predicted landing rows; after a replay the next kBandSkip windows store
// every row.
constexpr int kBandMargin = 1;
constexpr int kBandSkip = 8;

}  // namespace

namespace {

template <typename T>
int dalloc(pic_handle* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
    if (e != cudaSuccess) return map_cuda(e);
    h->allocs.push_back(q);
    *p = (T*)q;
    return PIC_OK;
}

void free_all(pic_handle* h) {
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    if (h->status_host) cudaFreeHost(h->status_host);
    h->status_host = nullptr;
}

int read_status(pic_handle* h) {
    cudaError_t e = cudaMemcpyAsync(h->status_host, h->B.status, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return map_cuda(e);
    return map_dev(*h->status_host);
}

// Resets the per-launch synchronisation words of the cooperative window.
cudaError_t reset_coop(pic_handle* h) {
    const size_t Np1 = (size_t)h->dp.n_cells + 1;
    cudaError_t e = cudaMemsetAsync(h->B.Qring, 0, sizeof(unsigned long long) * 3 * 2 * Np1 * pic::kQPad, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->B.notdone, 0, sizeof(int) * 4, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->B.bar, 0, sizeof(unsigned int) * 64, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->B.K_out, 0, sizeof(long long), h->st);
    return e;
}

// Grows the pool of timing events to at least `count`.
cudaError_t ensure_events(pic_handle* h, int count) {
    if (count > 256) return cudaErrorNotReady;  // stop timing, not the step
    while ((int)h->ev.size() < count) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        h->ev.push_back(e);
    }
    return cudaSuccess;
}

// Sum of the timed window launches (after the stream has been synchronised).
void collect_window_ms(pic_handle* h) {
    double ms = 0.0;
    for (int k = 0; k + 1 < h->ev_used; k += 2) {
        float x = 0.f;
        if (cudaEventElapsedTime(&x, h->ev[k], h->ev[k + 1]) == cudaSuccess) ms += x;
    }
    h->window_ms = ms;
    h->window_n = h->ev_used / 2;
    if (h->acc_on) {
        h->acc_ms += ms;
        h->acc_n += h->window_n;
    }
}

// Phase-space sort of the storage order before a window (see sort.cu).
cudaError_t maybe_sort(pic_handle* h, long long step_index) {
    if (h->prm.sort_every <= 0 || step_index % h->prm.sort_every != 0) return cudaSuccess;
    if (h->prec) return pic::launch_phase_sort32(h->sort32, h->n, h->sm_count, h->st, &h->launches);
    return pic::launch_phase_sort(h->sort, h->n, h->sm_count, h->st, &h->launches);
}

int run_window(pic_handle* h, int mode, long long n_iter) {
    if (h->n == 0) return PIC_OK;
    cudaError_t e = cudaMemsetAsync(h->B.status, 0, sizeof(int), h->st);
    if (e != cudaSuccess) return map_cuda(e);
    const int T_known = (mode == pic::MODE_ETD && h->prm.periods_once) ? 1 : 0;
    h->ev_used = 0;
    bool banded = false;
    if (h->prm.field_model == PIC_FIELD_POISSON) {
        const long long reps = mode == pic::MODE_ETD ? n_iter : 1;
        for (long long s = 0; s < reps && e == cudaSuccess; ++s) {
            if (mode == pic::MODE_ETD) e = maybe_sort(h, h->n_steps + s);
            if (e == cudaSuccess) e = reset_coop(h);
            const bool timed = e == cudaSuccess && ensure_events(h, h->ev_used + 2) == cudaSuccess;
            if (timed) cudaEventRecord(h->ev[h->ev_used], h->st);
            // FP64 ETD windows store only the trajectory rows around the
            // landing rows predicted from the previous step's periods
            pic::DevParams dp = h->dp;
            dp.band_m = 0;
            if (mode == pic::MODE_ETD && !T_known && !h->prec && (h->have_periods || s > 0) &&
                h->prm.max_window_steps + 3 + 2 * kBandMargin < 4096) {
                if (h->band_skip > 0) {
                    --h->band_skip;
                } else {
                    dp.band_m = kBandMargin;
                    banded = true;
                }
            }
            if (e == cudaSuccess) {
                const long long nf = mode == pic::MODE_FINE ? n_iter : 0;
                if (h->prec)
                    e = pic::launch_window32_coop(dp, h->B32, h->L, mode, T_known, nf, h->st, &h->launches, h->Tin32);
                else
                    e = pic::launch_window_coop(dp, h->B, h->L, mode, T_known, nf, h->st, &h->launches, h->Tin);
            }
            if (timed) {
                cudaEventRecord(h->ev[h->ev_used + 1], h->st);
                h->ev_used += 2;
            }
        }
    } else {
        if (mode == pic::MODE_ETD) e = maybe_sort(h, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->B.K_out, 0, sizeof(long long), h->st);
        if (e == cudaSuccess) {
            const long long ni = mode == pic::MODE_PERIODS ? 0 : n_iter;
            if (h->prec)
                e = pic::launch_window32_local(h->dp, h->B32, mode, T_known, ni, h->block, h->sm_count, h->st,
                                               &h->launches, h->Tin32);
            else
                e = pic::launch_window_local(h->dp, h->B, mode, T_known, ni, h->block, h->sm_count, h->st,
                                             &h->launches, h->Tin);
        }
    }
    if (e != cudaSuccess) return map_cuda(e);
    const int rc = read_status(h);
    if (!rc && banded) {
        // a window whose landing rows fell outside the stored band replayed
        // itself with every row; after one, the next windows store every row
        int replays = 0;
        e = cudaMemcpyAsync(&replays, h->B.notdone + 4, sizeof(int), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return map_cuda(e);
        if (replays > h->band_replays) h->band_skip = kBandSkip;
        h->band_replays = replays;
    }
    collect_window_ms(h);
    if (h->acc_on && mode == pic::MODE_FINE) h->acc_fine += n_iter;
    return rc;
}


// Public-order (R, V) of the state into device arrays, and back from
// h->tmpR / h->tmpV (FP32 form: rounded to nearest binary32).
cudaError_t unpack_state(pic_handle* h, double* r, double* v) {
    if (h->prec) return pic::launch_unpack_perm32(h->B32.y, h->perm, h->n, r, v, h->sm_count, h->st, &h->launches);
    return pic::launch_unpack_perm(h->B.y, h->perm, h->n, r, v, h->sm_count, h->st, &h->launches);
}
cudaError_t pack_state(pic_handle* h) {
    if (h->prec)
        return pic::launch_pack_perm32(h->tmpR, h->tmpV, h->perm, h->n, h->B32.y, h->sm_count, h->st, &h->launches);
    return pic::launch_pack_perm(h->tmpR, h->tmpV, h->perm, h->n, h->B.y, h->sm_count, h->st, &h->launches);
}

// Allocation and initial state of the FP32 form (precision 1).  The
// synchronisation words (Qring, barrier, status) live in h->B and are
// shared with B32.
int init32(pic_handle* h, const double* r0, const double* v0, int ptr_kind) {
    const pic_params* p = &h->prm;
    const long long n = h->n;
    const size_t N = (size_t)n;
    const size_t Np1 = (size_t)p->n_cells + 1;
    const long long ld = pic::window32_row_stride(n);
    const size_t LD = (size_t)(ld > 0 ? ld : 128);
    const bool poisson = p->field_model == PIC_FIELD_POISSON;
    const bool need_traj = poisson || !p->periods_once;
    h->prec = 1;
    pic::WinBufs32& B = h->B32;
    std::memset(&B, 0, sizeof(B));
    B.ld = (long long)LD;
    int rc = PIC_OK;
#define ALLOC(ptr, cnt)                         \
    do {                                        \
        if (!rc) rc = dalloc(h, &(ptr), (cnt)); \
    } while (0)
    ALLOC(B.y, LD);
    ALLOC(B.tr, LD);
    if (poisson) ALLOC(B.ce, LD);
    ALLOC(B.t1, N);
    ALLOC(B.T, N);
    ALLOC(B.o, N);
    ALLOC(B.N, N);
    ALLOC(h->tmpR, N);
    ALLOC(h->tmpV, N);
    ALLOC(h->perm, N);
    ALLOC(h->rot32, (size_t)2 * p->steps_per_turn);
    if (p->sort_every > 0) {
        ALLOC(h->perm_alt, N);
        ALLOC(h->y32_alt, LD);
        ALLOC(h->skey, N);
        ALLOC(h->scount, pic::kSortBinsTotal);
        if (p->periods_once) ALLOC(h->Tin32_alt, N);
    }
    if (poisson) {
        ALLOC(h->B.Qring, 3 * 2 * Np1 * pic::kQPad);
        ALLOC(h->Qf, Np1);
        ALLOC(h->nout_f, 1);
        ALLOC(h->Ef, Np1);
        ALLOC(h->edges_f, 2);
    }
    if (need_traj) ALLOC(B.traj, (size_t)p->max_window_steps * LD);
    if (p->periods_once) ALLOC(h->Tin32, N);
    ALLOC(h->B.notdone, 5);
    ALLOC(h->B.bar, 64);
    ALLOC(h->B.status, 1);
    ALLOC(h->B.K_out, 1);
#undef ALLOC
    if (rc) return rc;
    B.Qring = h->B.Qring;
    B.notdone = h->B.notdone;
    B.bar = h->B.bar;
    B.status = h->B.status;
    B.K_out = h->B.K_out;
    if (poisson) {
        char* mem = nullptr;
        rc = dalloc(h, &mem, pic::scan_scratch_bytes(p->n_cells));
        if (rc) return rc;
        const int tiles = (p->n_cells + pic::kScanTile - 1) / pic::kScanTile;
        pic::scan_scratch_layout(p->n_cells, tiles, mem, &h->S);
    }
    {
        long long want = (n + 255) / 256;
        long long cap = (long long)h->sm_count * 4;
        h->mom_grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
        rc = dalloc(h, &h->part_d, (size_t)h->mom_grid * pic::kMomDoubles);
        if (!rc) rc = dalloc(h, &h->part_i, (size_t)h->mom_grid * pic::kMomInts);
        if (rc) return rc;
    }
    cudaError_t e = cudaMallocHost(&h->status_host, sizeof(int));
    if (e != cudaSuccess) return map_cuda(e);
    const std::vector<float2> rot = rotation_table(p->steps_per_turn);
    e = cudaMemcpyAsync(h->rot32, rot.data(), sizeof(float2) * rot.size(), cudaMemcpyHostToDevice, h->st);
    h->dp.rot = h->rot32;
    if (e == cudaSuccess) e = cudaMemsetAsync(B.y, 0, sizeof(float2) * LD, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.tr, 0, sizeof(unsigned int) * LD, h->st);
    if (e == cudaSuccess && h->y32_alt) e = cudaMemsetAsync(h->y32_alt, 0, sizeof(float2) * LD, h->st);
    if (e == cudaSuccess && n > 0) {
        e = cudaMemcpyAsync(h->tmpR, r0, sizeof(double) * N, kind_to(ptr_kind), h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->tmpV, v0, sizeof(double) * N, kind_to(ptr_kind), h->st);
        if (e == cudaSuccess) e = pic::launch_iota(h->perm, n, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess) e = pic::launch_pack_perm32(h->tmpR, h->tmpV, h->perm, n, B.y, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.T, 0, sizeof(pic::CTime) * N, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.o, 0, sizeof(pic::CTime) * N, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.N, 0, sizeof(int) * N, h->st);
    }
    if (e != cudaSuccess) return map_cuda(e);
    pic::SortBufs32& S = h->sort32;
    S.y = &h->B32.y;
    S.y_alt = &h->y32_alt;
    S.perm = &h->perm;
    S.perm_alt = &h->perm_alt;
    S.Tin = p->periods_once ? &h->Tin32 : nullptr;
    S.Tin_alt = p->periods_once ? &h->Tin32_alt : nullptr;
    S.key = h->skey;
    S.count = h->scount;
    if (poisson) {
        rc = map_cuda(pic::window32_prepare(h->dp, h->block, p->blocks_per_sm, h->sm_count, B.ld, &h->L));
        if (rc) return rc;
    }
    if (p->periods_once && n > 0) {
        // step 1 once, at initialisation (Sec. 4.1)
        rc = run_window(h, pic::MODE_PERIODS, 0);
        if (!rc) rc = map_cuda(cudaMemcpyAsync(h->Tin32, B.T, sizeof(pic::CTime) * N, cudaMemcpyDeviceToDevice, h->st));
        if (!rc) h->have_periods = 1;
        if (rc) return rc;
    }
    return map_cuda(cudaStreamSynchronize(h->st));
}

}  // namespace

extern "C" {

void pic_default_params(pic_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps = 0.01;
    p->dt = 0.1;
    p->field_model = PIC_FIELD_POISSON;
    p->fine_solver = PIC_FINE_LAWSON_RK4;
    p->steps_per_turn = 100;
    p->n_cells = 256;
    p->r_min = -4.0;
    p->r_max = 4.0;
    p->total_charge = 1.0;
    p->weight_fixed = 1ull << 32;
    p->max_window_steps = 300;
    p->periods_once = 0;
    p->precision = 0;
    p->block_size = 0;
    p->blocks_per_sm = 0;
    p->sort_every = 1;
    p->wait_limit_ns = 0;
}

const char* pic_strerror(int s) {
    switch (s) {
        case PIC_OK: return "ok";
        case PIC_ERR_INVALID_ARG: return "invalid argument";
        case PIC_ERR_CUDA: return "CUDA error or no usable CUDA device";
        case PIC_ERR_TIMEOUT: return "device-side wait exceeded its time limit";
        case PIC_ERR_OVERFLOW: return "fixed-point charge would overflow (n*W >= 2^62)";
        case PIC_ERR_UNSUPPORTED: return "unsupported request";
        case PIC_ERR_NO_MEMORY: return "device memory allocation failed";
        case PIC_ERR_TOO_LARGE: return "size exceeds the fixed scratch capacity of a no-allocation entry point";
        default: return "unknown status";
    }
}

int pic_init(const pic_params* p, int64_t n, const double* r0, const double* v0, int ptr_kind, void* stream,
             pic_handle** out) {
    if (!out) return PIC_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_params(p, false);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!r0 || !v0)) || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE))
        return PIC_ERR_INVALID_ARG;
    if (n > 2147483647ll) return PIC_ERR_UNSUPPORTED;
    if (p->field_model == PIC_FIELD_POISSON) {
        if (p->n_cells > pic::kMaxCellsWindow) return PIC_ERR_UNSUPPORTED;
        if ((double)n * (double)p->weight_fixed >= 4.611686018427388e18) return PIC_ERR_OVERFLOW;
    }
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;

    pic_handle* h = new (std::nothrow) pic_handle();
    if (!h) return PIC_ERR_NO_MEMORY;
    h->prm = *p;
    h->n = n;
    h->st = (cudaStream_t)stream;
    h->sm_count = sms;
    make_devparams(p, n, &h->dp);
    h->block = p->block_size ? p->block_size : (p->field_model == PIC_FIELD_POISSON ? 1024 : 128);

    if (p->precision == 1) {
        rc = init32(h, r0, v0, ptr_kind);
        if (rc) {
            free_all(h);
            delete h;
            return rc;
        }
        *out = h;
        return PIC_OK;
    }

    const size_t N = (size_t)n;
    const size_t Np1 = (size_t)p->n_cells + 1;
    const bool need_traj = p->field_model == PIC_FIELD_POISSON || !p->periods_once;
    pic::WinBufs& B = h->B;
    std::memset(&B, 0, sizeof(B));
    cudaError_t e = cudaSuccess;
    rc = PIC_OK;
#define ALLOC(ptr, cnt)                         \
    do {                                        \
        if (!rc) rc = dalloc(h, &(ptr), (cnt)); \
    } while (0)
    ALLOC(B.y, N);
    ALLOC(B.t1, N);
    ALLOC(B.vp, N);
    ALLOC(B.T, N);
    ALLOC(B.o, N);
    ALLOC(B.N, N);
    ALLOC(B.tr, N);
    ALLOC(h->tmpR, N);
    ALLOC(h->tmpV, N);
    ALLOC(h->perm, N);
    if (p->sort_every > 0) {
        ALLOC(h->perm_alt, N);
        ALLOC(h->y_alt, N);
        ALLOC(h->skey, N);
        ALLOC(h->scount, pic::kSortBinsTotal);
        if (p->periods_once) ALLOC(h->Tin_alt, N);
    }
    if (p->field_model == PIC_FIELD_POISSON) {
        ALLOC(B.ce, N);
        ALLOC(B.ca, N);
        if (p->fine_solver == PIC_FINE_LAWSON_RK4) {
            ALLOC(B.cxr, N);
        } else {
            ALLOC(B.cx, N);
        }
        ALLOC(B.cj, N);
        ALLOC(B.Qring, 3 * 2 * Np1 * pic::kQPad);
        ALLOC(h->Qf, Np1);
        ALLOC(h->nout_f, 1);
        ALLOC(h->Ef, Np1);
        ALLOC(h->edges_f, 2);
    }
    if (need_traj) ALLOC(B.traj, ((size_t)p->max_window_steps + 1) * N);
    if (p->periods_once) ALLOC(h->Tin, N);
    ALLOC(B.notdone, 5);
    ALLOC(B.bar, 64);
    ALLOC(B.status, 1);
    ALLOC(B.K_out, 1);
#undef ALLOC
    if (!rc && p->field_model == PIC_FIELD_POISSON) {
        size_t bytes = pic::scan_scratch_bytes(p->n_cells);
        char* mem = nullptr;
        rc = dalloc(h, &mem, bytes);
        if (!rc) {
            int tiles = (p->n_cells + pic::kScanTile - 1) / pic::kScanTile;
            pic::scan_scratch_layout(p->n_cells, tiles, mem, &h->S);
        }
    }
    if (!rc) {
        long long want = (n + 255) / 256;
        long long cap = (long long)sms * 4;
        h->mom_grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
        rc = dalloc(h, &h->part_d, (size_t)h->mom_grid * pic::kMomDoubles);
        if (!rc) rc = dalloc(h, &h->part_i, (size_t)h->mom_grid * pic::kMomInts);
    }
    if (!rc) {
        e = cudaMallocHost(&h->status_host, sizeof(int));
        rc = map_cuda(e);
    }
    if (!rc && n > 0) {
        e = cudaMemcpyAsync(h->tmpR, r0, sizeof(double) * N, kind_to(ptr_kind), h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->tmpV, v0, sizeof(double) * N, kind_to(ptr_kind), h->st);
        if (e == cudaSuccess) e = pic::launch_pack(h->tmpR, h->tmpV, B.y, n, sms, h->st, &h->launches);
        if (e == cudaSuccess) e = pic::launch_iota(h->perm, n, sms, h->st, &h->launches);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.T, 0, sizeof(double) * N, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.o, 0, sizeof(double) * N, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.N, 0, sizeof(int) * N, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.tr, 0, sizeof(int2) * N, h->st);
        rc = map_cuda(e);
    }
    if (!rc) rc = map_cuda(cudaMemsetAsync(B.notdone, 0, sizeof(int) * 5, h->st));
    if (!rc) {
        pic::SortBufs& S = h->sort;
        S.y = &h->B.y;
        S.y_alt = &h->y_alt;
        S.perm = &h->perm;
        S.perm_alt = &h->perm_alt;
        S.Tin = p->periods_once ? &h->Tin : nullptr;
        S.Tin_alt = p->periods_once ? &h->Tin_alt : nullptr;
        S.key = h->skey;
        S.count = h->scount;
    }
    if (!rc && p->field_model == PIC_FIELD_POISSON)
        rc = map_cuda(pic::window_prepare(h->dp, h->block, p->blocks_per_sm, sms, &h->L));
    if (!rc && p->periods_once && n > 0) {
        // step 1 once, at initialisation (Sec. 4.1)
        rc = run_window(h, pic::MODE_PERIODS, 0);
        if (!rc) rc = map_cuda(cudaMemcpyAsync(h->Tin, B.T, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->st));
        if (!rc) h->have_periods = 1;
    }
    if (!rc) rc = map_cuda(cudaStreamSynchronize(h->st));
    if (rc) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return PIC_OK;
}

int pic_step(pic_handle* h, int64_t n_steps) {
    if (!h || n_steps < 0) return PIC_ERR_INVALID_ARG;
    if (n_steps == 0) return PIC_OK;
    int rc = run_window(h, pic::MODE_ETD, n_steps);
    if (rc == PIC_OK) {
        h->t += (double)n_steps * h->prm.dt;
        h->n_steps += n_steps;
        h->have_periods = 1;
    }
    return rc;
}

int pic_step_learned(pic_handle* h, const pic_mlp* m, int64_t n_steps, float scale_R, float scale_V,
                     double drift_tol, int64_t* n_fallback) {
    if (!h || !m || n_steps < 0 || !(drift_tol >= 0.0) || !std::isfinite(scale_R) || !std::isfinite(scale_V))
        return PIC_ERR_INVALID_ARG;
    if (n_fallback) *n_fallback = 0;
    if (n_steps == 0 || h->n == 0) {
        if (n_steps > 0 && h->n == 0) {
            h->t += (double)n_steps * h->prm.dt;
            h->n_steps += n_steps;
        }
        return PIC_OK;
    }
    const bool poisson = h->prm.field_model == PIC_FIELD_POISSON;
    const size_t Np1 = (size_t)h->dp.n_cells + 1;
    const size_t state_bytes = (size_t)h->n * (h->prec ? sizeof(float2) : sizeof(double2));
    int rc = PIC_OK;
    if (!h->y_prev) {
        char* yp = nullptr;
        rc = dalloc(h, &yp, state_bytes);
        if (!rc) h->y_prev = yp;
        if (!rc) rc = dalloc(h, &h->n_fb, 1);
        if (!rc && poisson) rc = dalloc(h, &h->psi, Np1);
        if (!rc && poisson && h->prec) rc = dalloc(h, &h->psi_f, 3 * Np1);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemsetAsync(h->n_fb, 0, sizeof(unsigned long long), h->st);
    for (long long step = 0; step < n_steps && e == cudaSuccess && rc == PIC_OK; ++step) {
        // the storage order of this step, then y^n and the field at t_n
        e = maybe_sort(h, h->n_steps);
        void* state = h->prec ? (void*)h->B32.y : (void*)h->B.y;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->y_prev, state, state_bytes, cudaMemcpyDeviceToDevice, h->st);
        if (e == cudaSuccess && poisson) {
            e = h->prec ? pic::launch_deposit32(h->dp, (const float*)h->B32.y, h->n, 2, h->Qf, h->nout_f, h->st,
                                                h->sm_count, &h->launches)
                        : pic::launch_deposit(h->dp, (const double*)h->B.y, h->n, 2, h->Qf, h->nout_f, h->st,
                                              h->sm_count, &h->launches);
            if (e == cudaSuccess) e = pic::launch_poisson(h->dp, h->Qf, h->Ef, h->edges_f, h->S, h->st, &h->launches);
            if (e == cudaSuccess)
                e = pic::launch_psi_nodes(h->Ef, h->dp.n_cells, h->dp.hr, h->psi, h->st, &h->launches, h->psi_f);
        }
        if (e != cudaSuccess) break;
        // the plain improved-ETD step, in the order just fixed
        const int saved = h->prm.sort_every;
        h->prm.sort_every = 0;
        rc = run_window(h, pic::MODE_ETD, 1);
        h->prm.sort_every = saved;
        if (rc) break;
        pic::LearnedArgs A;
        std::memset(&A, 0, sizeof(A));
        A.y_prev = h->y_prev;
        A.y = state;
        A.n = h->n;
        A.prec = h->prec;
        const double phase = h->t / h->prm.eps;
        A.in_sin = (float)std::sin(phase);
        A.in_cos = (float)std::cos(phase);
        A.in_dt = (float)h->prm.dt;
        A.scale_R = scale_R;
        A.scale_V = scale_V;
        A.tol = drift_tol;
        A.field = h->prm.field_model;
        A.eps = h->prm.eps;
        if (poisson) {
            A.E = h->Ef;
            A.psi = h->psi;
            A.edges = h->edges_f;
            A.r_min = h->dp.r_min;
            A.hr = h->dp.hr;
            A.inv_hr = h->dp.inv_hr;
            A.n_cells = h->dp.n_cells;
        }
        A.n_fallback = h->n_fb;
        A.tab_f = h->psi_f;
        e = pic::launch_learned_apply(m, A, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess) {
            h->t += h->prm.dt;
            h->n_steps += 1;
            h->have_periods = 1;
        }
    }
    if (rc) return rc;
    if (e != cudaSuccess) return map_cuda(e);
    unsigned long long nfb = 0;
    e = cudaMemcpyAsync(&nfb, h->n_fb, sizeof(nfb), cudaMemcpyDeviceToHost, h->st);
    if (e != cudaSuccess) return map_cuda(e);
    if ((rc = pic::mlp_take_error(m, h->st))) return rc;  // synchronises the stream: nfb has arrived
    if (n_fallback) *n_fallback = (int64_t)nfb;
    return PIC_OK;
}

// floor(t/h) fine steps and one step of the rest (FP64 path), time not advanced.
int fine_advance_raw(pic_handle* h, double t) {
    const long long nfull = (long long)std::floor(t / h->dp.h);
    const double rem = t - (double)nfull * h->dp.h;
    int rc = PIC_OK;
    if (nfull > 0) rc = run_window(h, pic::MODE_FINE, nfull);
    if (!rc && rem > 0.0) {
        const DevParams saved = h->dp;
        set_fine_step(&h->dp, h->prm.eps, rem);
        rc = run_window(h, pic::MODE_FINE, 1);
        h->dp = saved;
    }
    return rc;
}

int pic_fine_advance(pic_handle* h, double t) {
    if (!h || !(t >= 0.0) || !std::isfinite(t)) return PIC_ERR_INVALID_ARG;
    if (h->prec) return PIC_ERR_UNSUPPORTED;
    const int rc = fine_advance_raw(h, t);
    if (!rc) h->t += t;
    return rc;
}

int pic_step_classic(pic_handle* h, int64_t n_steps, int32_t period_mode, double* period, int64_t* fine_steps) {
    if (!h || n_steps < 0 || (period_mode != 0 && period_mode != 1)) return PIC_ERR_INVALID_ARG;
    if (h->prec) return PIC_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)h->n * sizeof(double2);
    int rc = PIC_OK;
    if (h->n > 0 && !h->y_prev) {
        char* yp = nullptr;
        rc = dalloc(h, &yp, bytes);
        if (rc) return rc;
        h->y_prev = yp;
    }
    std::vector<double> Th;
    h->acc_on = true;
    h->acc_ms = 0.0;
    h->acc_n = 0;
    h->acc_fine = 0;
    for (long long s = 0; s < n_steps && !rc; ++s) {
        double P = 2.0 * kPi * h->prm.eps;
        if (period_mode == 1 && h->n > 0) {
            // mean over the particles of their first-tour time (Remark
            // CompOfThePeriodsRem), summed in the public order
            const double* Tsrc = h->B.T;
            if (h->prm.periods_once) {
                Tsrc = h->Tin;
            } else {
                rc = run_window(h, pic::MODE_PERIODS, 0);
                if (rc) break;
            }
            Th.resize((size_t)h->n);
            long long K_det = 0;  // fine steps of the detection window
            cudaError_t e = pic::launch_permute_d(Tsrc, h->perm, h->n, 1.0, 1, h->tmpR, h->sm_count, h->st, &h->launches);
            if (e == cudaSuccess) e = cudaMemcpyAsync(Th.data(), h->tmpR, sizeof(double) * Th.size(), cudaMemcpyDeviceToHost, h->st);
            if (e == cudaSuccess && !h->prm.periods_once)
                e = cudaMemcpyAsync(&K_det, h->B.K_out, sizeof(long long), cudaMemcpyDeviceToHost, h->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
            h->acc_fine += K_det;
            if (e != cudaSuccess) {
                rc = map_cuda(e);
                break;
            }
            double sum = 0.0;
            for (double x : Th) sum += x;
            P = (sum / (double)h->n) * h->dp.h;
        }
        if (period) *period = P;
        const double o = std::fmod(h->prm.dt, P);
        const double N = std::rint((h->prm.dt - o) / P);
        if (h->n > 0) {
            cudaError_t e = cudaMemcpyAsync(h->y_prev, h->B.y, bytes, cudaMemcpyDeviceToDevice, h->st);
            if (e != cudaSuccess) {
                rc = map_cuda(e);
                break;
            }
            // y(t_n + P), then y(t_n + N P) = y_n + N (y(t_n + P) - y_n), then the rest o
            rc = period_mode == 0 ? run_window(h, pic::MODE_FINE, h->prm.steps_per_turn) : fine_advance_raw(h, P);
            if (rc) break;
            e = pic::launch_extrapolate_classic(h->B.y, (const double2*)h->y_prev, h->n, N, h->sm_count, h->st,
                                                &h->launches);
            if (e != cudaSuccess) {
                rc = map_cuda(e);
                break;
            }
            rc = fine_advance_raw(h, o);
            if (rc) break;
        }
        h->t += h->prm.dt;
        h->n_steps += 1;
    }
    h->acc_on = false;
    h->window_ms = h->acc_ms;
    h->window_n = h->acc_n;
    if (fine_steps) *fine_steps = h->acc_fine;
    return rc;
}

int pic_fine_steps(pic_handle* h, int64_t n_fine) {
    if (!h || n_fine < 0) return PIC_ERR_INVALID_ARG;
    if (n_fine == 0) return PIC_OK;
    int rc = run_window(h, pic::MODE_FINE, n_fine);
    if (rc == PIC_OK) h->t += (double)n_fine * h->dp.h;
    return rc;
}

int pic_get_field(pic_handle* h, int64_t* Q, double* E, double* rE_edges, int64_t* n_out, int ptr_kind) {
    if (!h || h->prm.field_model != PIC_FIELD_POISSON) return PIC_ERR_INVALID_ARG;
    if (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE) return PIC_ERR_INVALID_ARG;
    if (h->n == 0) return PIC_ERR_INVALID_ARG;
    const size_t Np1 = (size_t)h->dp.n_cells + 1;
    cudaError_t e = h->prec ? pic::launch_deposit32(h->dp, (const float*)h->B32.y, h->n, 2, h->Qf, h->nout_f, h->st,
                                                    h->sm_count, &h->launches)
                            : pic::launch_deposit(h->dp, (const double*)h->B.y, h->n, 2, h->Qf, h->nout_f, h->st,
                                                  h->sm_count, &h->launches);
    if (e == cudaSuccess) e = pic::launch_poisson(h->dp, h->Qf, h->Ef, h->edges_f, h->S, h->st, &h->launches);
    if (e == cudaSuccess && Q) e = cudaMemcpyAsync(Q, h->Qf, sizeof(long long) * Np1, kind_from(ptr_kind), h->st);
    if (e == cudaSuccess && E) e = cudaMemcpyAsync(E, h->Ef, sizeof(double) * Np1, kind_from(ptr_kind), h->st);
    if (e == cudaSuccess && rE_edges)
        e = cudaMemcpyAsync(rE_edges, h->edges_f, sizeof(double) * 2, kind_from(ptr_kind), h->st);
    if (e == cudaSuccess && n_out) e = cudaMemcpyAsync(n_out, h->nout_f, sizeof(long long), kind_from(ptr_kind), h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->status_host, h->S.status, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return map_cuda(e);
    return map_dev(*h->status_host);
}

int pic_moments(pic_handle* h, pic_moments_t* out) {
    if (!h || !out) return PIC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->t = h->t;
    out->n_steps = h->n_steps;
    out->n_particles = h->n;
    if (h->n == 0) return PIC_OK;
    const int G = h->mom_grid;
    std::vector<double> pd((size_t)G * pic::kMomDoubles);
    std::vector<long long> pi((size_t)G * pic::kMomInts);
    long long Kw = 0;
    cudaError_t e = h->prec ? pic::launch_moments32(h->dp, h->B32, h->part_d, h->part_i, G, h->st, &h->launches)
                            : pic::launch_moments(h->dp, h->B, h->part_d, h->part_i, G, h->st, &h->launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pd.data(), h->part_d, sizeof(double) * pd.size(), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pi.data(), h->part_i, sizeof(long long) * pi.size(), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&Kw, h->B.K_out, sizeof(long long), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return map_cuda(e);
    double a[pic::kMomDoubles] = {0, 0, 0, 0, 0, 0, INFINITY, -INFINITY};
    long long b[pic::kMomInts] = {LLONG_MAX, LLONG_MIN, 0};
    for (int g = 0; g < G; ++g) {
        const double* x = &pd[(size_t)g * pic::kMomDoubles];
        const long long* y = &pi[(size_t)g * pic::kMomInts];
        for (int q = 0; q < 6; ++q) a[q] += x[q];
        a[6] = std::fmin(a[6], x[6]);
        a[7] = std::fmax(a[7], x[7]);
        b[0] = y[0] < b[0] ? y[0] : b[0];
        b[1] = y[1] > b[1] ? y[1] : b[1];
        b[2] += y[2];
    }
    const double n = (double)h->n, w = h->prm.total_charge / n, hh = h->dp.h;
    out->mean_R = a[0] / n;
    out->mean_V = a[1] / n;
    out->rms_R = std::sqrt(a[2] / n);
    out->rms_V = std::sqrt(a[3] / n);
    out->kinetic = w * 0.5 * (a[2] + a[3]);
    out->duffing_energy = w * (0.5 * (a[2] + a[3]) + 0.25 * h->prm.eps * a[4]);
    if (h->have_periods) {
        out->T_min = a[6] * hh;
        out->T_max = a[7] * hh;
        out->T_mean = a[5] / n * hh;
        out->N_min = b[0];
        out->N_max = b[1];
        out->n_no_period = b[2];
        out->window_steps = Kw;
    }
    out->window_ms = h->window_ms;
    out->window_launches = h->window_n;
    out->band_replays = h->band_replays;
    if (h->prm.field_model == PIC_FIELD_POISSON) {
        std::vector<int64_t> Q((size_t)h->dp.n_cells + 1);
        int64_t nout = 0;
        int rc = pic_get_field(h, Q.data(), nullptr, nullptr, &nout, PIC_PTR_HOST);
        if (rc) return rc;
        long long tot = 0;
        for (int64_t q : Q) tot += (long long)q;
        out->Q_total = tot;
        out->n_out_of_mesh = nout;
        out->charge = (double)tot * h->dp.q_unit + (double)nout * w;
    } else {
        out->charge = h->prm.total_charge;
    }
    return PIC_OK;
}

int pic_get_particles(pic_handle* h, double* r, double* v, int ptr_kind) {
    if (!h || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    if (h->n == 0) return PIC_OK;
    const size_t bytes = sizeof(double) * (size_t)h->n;
    cudaError_t e;
    double* dr = ptr_kind == PIC_PTR_DEVICE ? r : h->tmpR;
    double* dv = ptr_kind == PIC_PTR_DEVICE ? v : h->tmpV;
    e = unpack_state(h, dr, dv);
    if (ptr_kind == PIC_PTR_HOST) {
        if (e == cudaSuccess && r) e = cudaMemcpyAsync(r, h->tmpR, bytes, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, h->tmpV, bytes, cudaMemcpyDeviceToHost, h->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return map_cuda(e);
}

int pic_set_particles(pic_handle* h, const double* r, const double* v, int ptr_kind) {
    if (!h || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    if (h->n == 0) return PIC_OK;
    if (!r || !v) return PIC_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)h->n;
    cudaError_t e = cudaMemcpyAsync(h->tmpR, r, bytes, kind_to(ptr_kind), h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tmpV, v, bytes, kind_to(ptr_kind), h->st);
    if (e == cudaSuccess) e = pack_state(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return map_cuda(e);
}

int pic_get_periods(pic_handle* h, double* T, int64_t* N, double* o, int ptr_kind) {
    if (!h || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    if (h->n == 0) return PIC_OK;
    const size_t n = (size_t)h->n;
    cudaError_t e = cudaSuccess;
    double *dT = T, *dO = o;
    long long* dN = (long long*)N;
    void* tmp = nullptr;
    if (ptr_kind == PIC_PTR_HOST) {
        e = cudaMallocAsync(&tmp, n * (2 * sizeof(double) + sizeof(long long)), h->st);
        if (e != cudaSuccess) return map_cuda(e);
        dT = (double*)tmp;
        dO = (double*)tmp + n;
        dN = (long long*)((double*)tmp + 2 * n);
    }
    // per-slot results to the public order, in units of time
    if (h->prec) {
        if (T) e = pic::launch_ctime_out(h->B32.T, h->perm, h->n, h->dp.h, dT, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess && o) e = pic::launch_ctime_out(h->B32.o, h->perm, h->n, h->dp.h, dO, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess && N) e = pic::launch_scatter_i(h->B32.N, h->perm, h->n, dN, h->sm_count, h->st, &h->launches);
    } else {
        if (T) e = pic::launch_permute_d(h->B.T, h->perm, h->n, h->dp.h, 1, dT, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess && o) e = pic::launch_permute_d(h->B.o, h->perm, h->n, h->dp.h, 1, dO, h->sm_count, h->st, &h->launches);
        if (e == cudaSuccess && N) e = pic::launch_scatter_i(h->B.N, h->perm, h->n, dN, h->sm_count, h->st, &h->launches);
    }
    if (ptr_kind == PIC_PTR_HOST) {
        if (e == cudaSuccess && T) e = cudaMemcpyAsync(T, dT, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess && o) e = cudaMemcpyAsync(o, dO, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess && N) e = cudaMemcpyAsync(N, dN, n * sizeof(long long), cudaMemcpyDeviceToHost, h->st);
        cudaError_t e2 = cudaFreeAsync(tmp, h->st);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return map_cuda(e);
}

int pic_get_state(pic_handle* h, pic_state_t* out) {
    if (!h || !out) return PIC_ERR_INVALID_ARG;
    out->t = h->t;
    out->n_steps = h->n_steps;
    if (h->n == 0) return PIC_OK;
    if (!out->r || !out->v || !out->T) return PIC_ERR_INVALID_ARG;
    const size_t n = (size_t)h->n;
    cudaError_t e = unpack_state(h, h->tmpR, h->tmpV);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->r, h->tmpR, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->v, h->tmpV, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) {
        if (h->prec) {
            const pic::CTime* Ts = h->prm.periods_once ? h->Tin32 : h->B32.T;
            e = pic::launch_ctime_out(Ts, h->perm, h->n, 1.0, h->tmpR, h->sm_count, h->st, &h->launches);
        } else {
            const double* Ts = h->prm.periods_once ? h->Tin : h->B.T;
            e = pic::launch_permute_d(Ts, h->perm, h->n, 1.0, 1, h->tmpR, h->sm_count, h->st, &h->launches);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->T, h->tmpR, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return map_cuda(e);
}

int pic_set_state(pic_handle* h, const pic_state_t* in) {
    if (!h || !in) return PIC_ERR_INVALID_ARG;
    if (h->n > 0 && (!in->r || !in->v || !in->T)) return PIC_ERR_INVALID_ARG;
    if (in->n_steps < 0) return PIC_ERR_INVALID_ARG;
    const size_t n = (size_t)h->n;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(h->tmpR, in->r, n * sizeof(double), cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->tmpV, in->v, n * sizeof(double), cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = pack_state(h);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->tmpR, in->T, n * sizeof(double), cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) {
            if (h->prec) {
                pic::CTime* Ts = h->prm.periods_once ? h->Tin32 : h->B32.T;
                e = pic::launch_ctime_in(h->tmpR, h->perm, h->n, Ts, h->sm_count, h->st, &h->launches);
            } else {
                double* Ts = h->prm.periods_once ? h->Tin : h->B.T;
                e = pic::launch_permute_d(h->tmpR, h->perm, h->n, 1.0, 0, Ts, h->sm_count, h->st, &h->launches);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    }
    if (e != cudaSuccess) return map_cuda(e);
    h->t = in->t;
    h->n_steps = in->n_steps;
    return PIC_OK;
}

int pic_window_time(const pic_handle* h, double* ms, int64_t* launches) {
    if (!h) return PIC_ERR_INVALID_ARG;
    if (ms) *ms = h->window_ms;
    if (launches) *launches = h->window_n;
    return PIC_OK;
}

int64_t pic_num_particles(const pic_handle* h) { return h ? h->n : -1; }

int64_t pic_launch_count(const pic_handle* h) { return h ? h->launches : -1; }

void pic_destroy(pic_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
}

// ---------------------------------------------------------- standalone mesh

int pic_deposit(const pic_params* p, int64_t n, const double* R_dev, int64_t* Q_dev, int64_t* n_out_dev,
                void* stream) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !R_dev) || !Q_dev || !n_out_dev) return PIC_ERR_INVALID_ARG;
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;
    DevParams d;
    make_devparams(p, n, &d);
    return map_cuda(pic::launch_deposit(d, R_dev, n, 1, (long long*)Q_dev, (long long*)n_out_dev,
                                        (cudaStream_t)stream, sms, nullptr));
}

int pic_deposit_f32(const pic_params* p, int64_t n, const float* R_dev, int64_t* Q_dev, int64_t* n_out_dev,
                    void* stream) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !R_dev) || !Q_dev || !n_out_dev) return PIC_ERR_INVALID_ARG;
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;
    DevParams d;
    make_devparams(p, n, &d);
    return map_cuda(pic::launch_deposit32(d, R_dev, n, 1, (long long*)Q_dev, (long long*)n_out_dev,
                                          (cudaStream_t)stream, sms, nullptr));
}

}  // extern "C"

// Shared body of pic_poisson and pic_poisson_noalloc: S is the caller's
// scratch (flags, tile counter and status are cleared here, on the stream).
int pic::poisson_with_scratch(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                              double* rE_edges_dev, const pic::ScanScratch* S, void* stream) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (n_particles <= 0 || !Q_dev || !E_dev || !rE_edges_dev || !S) return PIC_ERR_INVALID_ARG;
    if ((double)n_particles * (double)p->weight_fixed >= 4.611686018427388e18) return PIC_ERR_OVERFLOW;
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;
    DevParams d;
    make_devparams(p, n_particles, &d);
    cudaStream_t st = (cudaStream_t)stream;
    int status = 0;
    cudaError_t e = pic::launch_poisson(d, (const long long*)Q_dev, E_dev, rE_edges_dev, *S, st, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, S->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return map_cuda(e);
    return map_dev(status);
}

extern "C" {

int pic_poisson(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                double* rE_edges_dev, void* stream) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (n_particles <= 0 || !Q_dev || !E_dev || !rE_edges_dev) return PIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int tiles = (p->n_cells + pic::kScanTile - 1) / pic::kScanTile;
    const size_t bytes = pic::scan_scratch_layout(p->n_cells, tiles, nullptr, nullptr);
    void* mem = nullptr;
    cudaError_t e = cudaMallocAsync(&mem, bytes, st);
    if (e != cudaSuccess) return map_cuda(e);
    pic::ScanScratch S;
    pic::scan_scratch_layout(p->n_cells, tiles, mem, &S);
    rc = pic::poisson_with_scratch(p, n_particles, Q_dev, E_dev, rE_edges_dev, &S, stream);
    e = cudaFreeAsync(mem, st);
    if (rc == PIC_OK && e != cudaSuccess) rc = map_cuda(e);
    return rc;
}

int pic_gather(const pic_params* p, int64_t n, const double* R_dev, const double* E_dev,
               const double* rE_edges_dev, double* e_dev, void* stream) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!R_dev || !e_dev)) || !E_dev || !rE_edges_dev) return PIC_ERR_INVALID_ARG;
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;
    DevParams d;
    make_devparams(p, n, &d);
    return map_cuda(pic::launch_gather(d, R_dev, n, E_dev, rE_edges_dev, e_dev, (cudaStream_t)stream, sms, nullptr));
}

int pic_frozen_potential(const pic_params* p, const double* E_dev, const double* rE_edges_dev, double* psi_nodes_dev,
                         int64_t n, const double* R_dev, double* psi_dev, void* stream) {
    int rc = check_params(p, false);
    if (rc) return rc;
    const bool poisson = p->field_model == PIC_FIELD_POISSON;
    if (n < 0 || (n > 0 && (!R_dev || !psi_dev))) return PIC_ERR_INVALID_ARG;
    if (poisson && (!E_dev || !rE_edges_dev || !psi_nodes_dev)) return PIC_ERR_INVALID_ARG;
    int sms = 0;
    if ((rc = current_sm_count(&sms))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    pic::LearnedArgs A;
    std::memset(&A, 0, sizeof(A));
    A.n = n;
    A.field = p->field_model;
    A.eps = p->eps;
    cudaError_t e = cudaSuccess;
    if (poisson) {
        DevParams d;
        make_devparams(p, 1, &d);
        e = pic::launch_psi_nodes(E_dev, d.n_cells, d.hr, psi_nodes_dev, st, nullptr);
        A.E = E_dev;
        A.psi = psi_nodes_dev;
        A.edges = rE_edges_dev;
        A.r_min = d.r_min;
        A.hr = d.hr;
        A.inv_hr = d.inv_hr;
        A.n_cells = d.n_cells;
    }
    if (e == cudaSuccess) e = pic::launch_psi_eval(A, R_dev, psi_dev, sms, st);
    return map_cuda(e);
}

// Testing hook: a Poisson window whose grid barrier waits for one arrival
// that never comes, with the given limit; returns the status pic_step gives.
int pic_test_barrier_timeout(int64_t wait_limit_ns, int32_t precision, void* stream) {
    if (wait_limit_ns <= 0 || wait_limit_ns > 10000000000ll) return PIC_ERR_INVALID_ARG;
    if (precision != 0 && precision != 1) return PIC_ERR_INVALID_ARG;
    pic_params p;
    pic_default_params(&p);
    p.wait_limit_ns = wait_limit_ns;
    p.precision = precision;
    p.block_size = 128;
    std::vector<double> r(256), v(256);
    for (int i = 0; i < 256; ++i) {
        r[i] = -1.0 + 2.0 * (i + 0.5) / 256.0;
        v[i] = 0.5;
    }
    pic_handle* h = nullptr;
    int rc = pic_init(&p, 256, r.data(), v.data(), PIC_PTR_HOST, stream, &h);
    if (rc) return rc;
    h->dp.bar_extra = 1;
    rc = pic_step(h, 1);
    pic_destroy(h);
    return rc;
}

}  // extern "C"

// ------------------------------------------------------------ batched form

struct pic_batch {
    std::vector<pic_handle*> hs;
    cudaStream_t st = nullptr;
    int sm_count = 0;
    int n = 0;
    pic::BeamDesc32* d_desc = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;  // pinned
    unsigned long long* d_times = nullptr;  // per beam: first start, last end of its blocks (ns)
    unsigned long long* h_times = nullptr;  // pinned copy
    std::vector<pic::BeamDesc32> desc;
    int block = 1024, bps = 1, grid = 0, sort_every = 4, copies = 1;
    double alloc_power = 1.0;
    bool shares_measured = false;  // block shares from measured beam times (pic_batch_tune)
    size_t smem = 0;
    int max_cells = 0;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = false, use_graph = true;
    cudaError_t graph_error = cudaSuccess;
    // the graph is captured on and replayed from a stream of the batch's own
    // (the caller's stream may be the legacy default stream, which cannot be
    // captured), ordered after the caller's work by an event
    cudaStream_t gst = nullptr;
    cudaEvent_t ev_in = nullptr;
    long long steps = 0, launches = 0;
};

namespace {

void batch_drop_graph(pic_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_ok = false;
}

// Descriptors of the current buffers (the sort swaps them) and launch shape.
cudaError_t batch_upload(pic_batch* b) {
    for (int i = 0; i < b->n; ++i) {
        pic_handle* h = b->hs[i];
        pic::BeamDesc32& d = b->desc[i];
        d.P = h->dp;
        // the batch's shared memory is sized for b->copies copies of the
        // largest mesh; a beam with a smaller mesh takes up to four where
        // they fit, while its blocks still deposit at least 2048 positions
        // per copy and cycle (more copies spread same-cell atomics)
        int cp = b->copies;
        if (h->prm.field_model == PIC_FIELD_POISSON && d.n_blocks > 0) {
            const long long per_block = (h->n + d.n_blocks - 1) / d.n_blocks;
            while (cp < 4 && pic::window32_batch_smem(h->prm.n_cells, 2 * cp) <= b->smem &&
                   per_block >= 2048ll * 2 * cp)
                cp *= 2;
        }
        d.P.hist_copies = cp;
        d.B = h->B32;
        d.Tin = h->prm.periods_once ? h->Tin32 : nullptr;
        d.T_known = h->prm.periods_once ? 1 : 0;
        d.coop = h->prm.field_model == PIC_FIELD_POISSON ? 1 : 0;
        d.t_ns = b->d_times + 2 * i;
    }
    batch_drop_graph(b);
    return cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(pic::BeamDesc32) * b->n, cudaMemcpyHostToDevice, b->st);
}

// Blocks per beam that minimise the largest predicted window (min-max
// greedy), on plain arrays.  Beam i (coop[i]: Poisson, else an analytic
// field; np[i] particles) took ms[i] on blocks_meas[i] blocks of
// block_meas threads.  A Poisson beam's window is predicted as
// ms n_0 / n on n blocks (its sweeps divide over the blocks); an analytic
// beam's as ms r(n) / r(n_0), r(n) = ceil(np / (n block)) being the
// particles one thread advances one after the other.  Every beam starts at
// its least share lo[i]; then the beam with the largest prediction that
// more blocks would shorten gets them (one block, or for an analytic beam
// the blocks that take r one lower), within need[i] and the grid G, until
// the grid is used up or no beam can be shortened.  false: the least
// shares exceed G.
static bool shares_minmax_core(int n, const char* coop, const long long* np, const double* ms,
                               const long long* blocks_meas, int block_meas, int block, long long G,
                               const long long* lo, const long long* need, long long* nb) {
    auto rounds = [&](int i, long long m, int blk) { return (np[i] + m * blk - 1) / (m * blk); };
    auto pred = [&](int i, long long m) -> double {
        const double t = std::max(ms[i], 1e-6);
        if (coop[i]) return t * (double)blocks_meas[i] / (double)m;
        return t * (double)rounds(i, m, block) / (double)rounds(i, blocks_meas[i], block_meas);
    };
    long long used = 0;
    for (int i = 0; i < n; ++i) {
        nb[i] = lo[i];
        used += nb[i];
    }
    if (used > G) return false;
    for (;;) {
        int best = -1;
        long long best_to = 0;
        double best_p = -1.0;
        for (int i = 0; i < n; ++i) {
            if (nb[i] >= need[i]) continue;
            long long to = nb[i] + 1;
            if (!coop[i]) {
                // fewest blocks with one round less
                const long long r = rounds(i, nb[i], block);
                to = r > 1 ? (np[i] + (r - 1) * block - 1) / ((r - 1) * block) : need[i];
                if (to > need[i]) to = need[i];
                if (to <= nb[i]) to = nb[i] + 1;
            }
            if (used + (to - nb[i]) > G) continue;
            const double p = pred(i, nb[i]);
            if (p > best_p) {
                best = i;
                best_p = p;
                best_to = to;
            }
        }
        if (best < 0) break;
        used += best_to - nb[best];
        nb[best] = best_to;
    }
    return true;
}

// Measured windows of the beams: beam i took ms[i] on blocks[i] blocks of
// `block` threads.
struct BeamTimes {
    std::vector<double> ms;
    std::vector<long long> blocks;
    int block = 0;
};

// shares_minmax_core for the beams of a batch.
static bool shares_minmax(const pic_batch* b, const BeamTimes& t, int block, long long G,
                          const std::vector<long long>& lo, const std::vector<long long>& need,
                          std::vector<long long>& nb) {
    const int n = b->n;
    std::vector<char> coop(n);
    std::vector<long long> np(n);
    for (int i = 0; i < n; ++i) {
        coop[i] = b->hs[i]->prm.field_model == PIC_FIELD_POISSON;
        np[i] = b->hs[i]->n > 0 ? b->hs[i]->n : 1;
    }
    return shares_minmax_core(n, coop.data(), np.data(), t.ms.data(), t.blocks.data(), t.block, block, G, lo.data(),
                              need.data(), nb.data());
}

// Blocks per beam in proportion to (its particles)^power, at least one and
// at most what its particles fill; weight 1/4 for the analytic fields (no
// field cycle).  meas (may be null): shares from the beams' measured
// windows instead (shares_minmax).
int batch_configure(pic_batch* b, int block, int bps_want, double power, int copies,
                    const BeamTimes* meas = nullptr) {
    if (block < 128 || block > 1024 || (block & 31)) return PIC_ERR_INVALID_ARG;
    if (copies != 1 && copies != 2 && copies != 4) return PIC_ERR_INVALID_ARG;
    const size_t smem = pic::window32_batch_smem(b->max_cells, copies);
    if (smem > 227 * 1024) return PIC_ERR_UNSUPPORTED;
    if (smem > 0) {
        // the larger of the new and the current size, so that the current
        // configuration stays launchable if this one is refused below
        cudaError_t e = pic::window32_batch_attr(smem > b->smem ? smem : b->smem);
        if (e != cudaSuccess) return map_cuda(e);
    }
    int bps = 0;
    cudaError_t e = pic::window32_batch_occupancy(block, smem, &bps);
    if (e != cudaSuccess) return map_cuda(e);
    if (bps < 1) return PIC_ERR_UNSUPPORTED;
    if (bps_want > 0 && bps_want < bps) bps = bps_want;
    const long long G = (long long)bps * b->sm_count;
    if (G < b->n) return PIC_ERR_UNSUPPORTED;
    std::vector<double> w(b->n);
    std::vector<long long> need(b->n), lo(b->n), nb(b->n);
    double wsum = 0.0;
    for (int i = 0; i < b->n; ++i) {
        pic_handle* h = b->hs[i];
        const bool coop = h->prm.field_model == PIC_FIELD_POISSON;
        const long long groups = (h->B32.ld + 127) / 128;
        need[i] = coop ? (groups + block / 32 - 1) / (block / 32) : (h->n + block - 1) / block;
        if (need[i] < 1) need[i] = 1;
        // a Poisson beam's blocks deposit at most 2^21 positions each per cycle
        lo[i] = coop ? std::max(1ll, (groups * 128 + (1ll << 21) - 1) >> 21) : 1;
        if (lo[i] > need[i]) need[i] = lo[i];
        w[i] = (coop ? 1.0 : 0.25) * std::pow((double)(h->n > 0 ? h->n : 1), power);
        wsum += w[i];
    }
    if (meas && (int)meas->ms.size() == b->n && (int)meas->blocks.size() == b->n && meas->block > 0) {
        if (!shares_minmax(b, *meas, block, G, lo, need, nb)) return PIC_ERR_UNSUPPORTED;
    } else {
        meas = nullptr;
        long long used = 0;
        for (int i = 0; i < b->n; ++i) {
            long long k = (long long)std::floor((double)(G - b->n) * w[i] / wsum) + 1;
            nb[i] = k < need[i] ? k : need[i];
            used += nb[i];
        }
        // hand out what is left, largest deficit first
        while (used < G) {
            int best = -1;
            double bestd = 0.0;
            for (int i = 0; i < b->n; ++i) {
                if (nb[i] >= need[i]) continue;
                const double d = (double)G * w[i] / wsum - (double)nb[i];
                if (best < 0 || d > bestd) {
                    best = i;
                    bestd = d;
                }
            }
            if (best < 0) break;
            ++nb[best];
            ++used;
        }
    }
    int first = 0;
    for (int i = 0; i < b->n; ++i) {
        pic_handle* h = b->hs[i];
        if (h->prm.field_model == PIC_FIELD_POISSON) {
            const long long groups = (h->B32.ld + 127) / 128;
            if ((groups + nb[i] - 1) / nb[i] * 128 > (1ll << 21)) return PIC_ERR_UNSUPPORTED;
        }
        b->desc[i].first_block = first;
        b->desc[i].n_blocks = (int)nb[i];
        first += (int)nb[i];
    }
    b->grid = first;
    b->block = block;
    b->bps = bps;
    b->alloc_power = power;
    b->shares_measured = meas != nullptr;
    b->copies = copies;
    b->smem = smem;
    return map_cuda(batch_upload(b));
}

cudaError_t batch_enqueue_step(pic_batch* b, cudaStream_t st) {
    cudaError_t e = pic::launch_batch_reset(b->d_desc, b->n, st);
    if (e == cudaSuccess) e = pic::launch_window32_batch(b->d_desc, b->n, b->grid, b->block, b->smem, st);
    if (e == cudaSuccess) e = pic::launch_batch_status(b->d_desc, b->n, b->d_status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_times, b->d_times, sizeof(unsigned long long) * 2 * b->n, cudaMemcpyDeviceToHost, st);
    return e;
}

// One macro step of every beam: sorts when due, then the captured graph of
// reset + cooperative window + status gather (captured again after a sort
// has moved buffers).
int batch_one_step(pic_batch* b) {
    cudaError_t e = cudaSuccess;
    if (b->sort_every > 0 && b->steps % b->sort_every == 0) {
        for (int i = 0; i < b->n && e == cudaSuccess; ++i)
            if (b->hs[i]->n > 0) e = pic::launch_phase_sort32(b->hs[i]->sort32, b->hs[i]->n, b->sm_count, b->st, &b->launches);
        if (e == cudaSuccess) e = batch_upload(b);
    }
    if (e == cudaSuccess && b->use_graph && !b->graph_ok) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->gst, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = batch_enqueue_step(b, b->gst);
            const cudaError_t e2 = cudaStreamEndCapture(b->gst, &g);
            e = e1 != cudaSuccess ? e1 : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            b->graph_ok = true;
        } else {
            // capture is not available here: launch the same work directly
            b->graph_error = e;
            cudaGetLastError();
            b->use_graph = false;
            e = cudaSuccess;
        }
    }
    if (e == cudaSuccess) {
        if (b->use_graph) {
            e = cudaEventRecord(b->ev_in, b->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->gst, b->ev_in, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->gst);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->gst);
        } else {
            e = batch_enqueue_step(b, b->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        }
    }
    if (e != cudaSuccess) return map_cuda(e);
    b->launches += 3;
    for (int i = 0; i < b->n; ++i)
        if (b->h_status[i] != pic::DEV_OK) return map_dev(b->h_status[i]);
    for (int i = 0; i < b->n; ++i) {
        pic_handle* h = b->hs[i];
        h->t += h->prm.dt;
        h->n_steps += 1;
        h->have_periods = 1;
        // the beam's window within the shared launch: first start to last end of its blocks
        const unsigned long long t0 = b->h_times[2 * i], t1 = b->h_times[2 * i + 1];
        h->window_ms = t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
        h->window_n = 1;
    }
    b->steps += 1;
    return PIC_OK;
}

void batch_free(pic_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->gst) cudaStreamSynchronize(b->gst);
    batch_drop_graph(b);
    if (b->gst) cudaStreamDestroy(b->gst);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    for (pic_handle* h : b->hs) pic_destroy(h);
    b->hs.clear();
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_status) cudaFree(b->d_status);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->d_times) cudaFree(b->d_times);
    if (b->h_times) cudaFreeHost(b->h_times);
    delete b;
}

}  // namespace

extern "C" {

int pic_batch_create(int32_t n_beams, const pic_params* params, const int64_t* n_particles, const double* const* r0,
                     const double* const* v0, void* stream, pic_batch** out) {
    if (!out || n_beams < 1 || n_beams > 4096 || !params || !n_particles || !r0 || !v0) return PIC_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n_beams; ++i) {
        if (params[i].precision != 1) return PIC_ERR_UNSUPPORTED;
        if (params[i].field_model == PIC_FIELD_POISSON && params[i].n_cells > pic::kMaxCellsWindow)
            return PIC_ERR_UNSUPPORTED;
    }
    int sms = 0;
    int rc = current_sm_count(&sms);
    if (rc) return rc;
    pic_batch* b = new (std::nothrow) pic_batch();
    if (!b) return PIC_ERR_NO_MEMORY;
    b->st = (cudaStream_t)stream;
    b->sm_count = sms;
    b->n = n_beams;
    b->desc.resize(n_beams);
    std::memset(b->desc.data(), 0, sizeof(pic::BeamDesc32) * n_beams);
    for (int i = 0; i < n_beams && !rc; ++i) {
        pic_params p = params[i];
        p.sort_every = 1;  // sort buffers exist; the batch decides when to sort
        pic_handle* h = nullptr;
        rc = pic_init(&p, n_particles[i], r0[i], v0[i], PIC_PTR_HOST, stream, &h);
        if (!rc) {
            b->hs.push_back(h);
            if (p.field_model == PIC_FIELD_POISSON && p.n_cells > b->max_cells) b->max_cells = p.n_cells;
        }
    }
    if (!rc) {
        cudaError_t e = cudaMalloc(&b->d_desc, sizeof(pic::BeamDesc32) * n_beams);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * n_beams);
        if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int) * n_beams);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_times, sizeof(unsigned long long) * 2 * n_beams);
        if (e == cudaSuccess) e = cudaMallocHost(&b->h_times, sizeof(unsigned long long) * 2 * n_beams);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gst, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
        rc = map_cuda(e);
    }
    if (!rc) rc = batch_configure(b, 1024, 1, 1.0, 1);
    if (!rc) rc = map_cuda(cudaStreamSynchronize(b->st));
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return PIC_OK;
}

int pic_batch_step(pic_batch* b, int64_t n_steps) {
    if (!b || n_steps < 0) return PIC_ERR_INVALID_ARG;
    for (int64_t s = 0; s < n_steps; ++s) {
        const int rc = batch_one_step(b);
        if (rc) return rc;
    }
    return PIC_OK;
}

int pic_batch_set_config(pic_batch* b, int32_t block, int32_t blocks_per_sm, double alloc_power, int32_t sort_every,
                         int32_t hist_copies) {
    if (!b || sort_every < 0 || !(alloc_power >= 0.0 && alloc_power <= 2.0)) return PIC_ERR_INVALID_ARG;
    const int rc = batch_configure(b, block, blocks_per_sm, alloc_power, hist_copies);
    if (!rc) b->sort_every = sort_every;
    return rc;
}

int pic_batch_get_config(const pic_batch* b, pic_batch_config_t* out) {
    if (!b || !out) return PIC_ERR_INVALID_ARG;
    out->block = b->block;
    out->blocks_per_sm = b->bps;
    out->grid = b->grid;
    out->sort_every = b->sort_every;
    out->alloc_power = b->alloc_power;
    out->graph = b->use_graph ? 1 : 0;
    out->graph_error = (int32_t)b->graph_error;
    out->hist_copies = b->copies;
    out->shares_measured = b->shares_measured ? 1 : 0;
    return PIC_OK;
}

int pic_batch_tune(pic_batch* b, int32_t steps_per_trial, pic_batch_config_t* best) {
    if (!b || steps_per_trial < 1) return PIC_ERR_INVALID_ARG;
    struct Cand {
        int block, bps;
        double power;
        int copies;
    };
    std::vector<Cand> shapes;
    const Cand base[] = {{1024, 1, 1.0, 1}, {1024, 1, 0.85, 1}, {512, 2, 1.0, 1}, {512, 2, 0.85, 1}, {256, 4, 1.0, 1}};
    for (int copies : {1, 2, 4})
        for (Cand c : base) {
            c.copies = copies;
            shapes.push_back(c);
        }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PIC_ERR_CUDA;
    std::vector<double> beam_ms(b->n);  // each beam's mean window time over the last trial
    // One trial: a step that captures and warms, then `steps` timed steps.
    // *ms: the mean step (sorts, graph captures and host work included);
    // *span: the mean launch span, first block start to last block end over
    // all beams (device timer), which is what launch shapes and block shares
    // change, without the sorts that fall into some trials and not others.
    auto trial = [&](int steps, double* ms, double* span) -> int {
        int rc = batch_one_step(b);  // capture and warm
        if (rc) return rc;
        std::fill(beam_ms.begin(), beam_ms.end(), 0.0);
        double sp = 0.0;
        cudaEventRecord(e0, b->st);
        for (int s = 0; s < steps && !rc; ++s) {
            rc = batch_one_step(b);
            unsigned long long lo = ~0ull, hi = 0ull;
            for (int i = 0; i < b->n; ++i) {
                beam_ms[i] += b->hs[i]->window_ms / steps;
                const unsigned long long t0 = b->h_times[2 * i], t1 = b->h_times[2 * i + 1];
                if (t1 > t0) {
                    lo = std::min(lo, t0);
                    hi = std::max(hi, t1);
                }
            }
            sp += hi > lo ? (double)(hi - lo) * 1e-6 / steps : 0.0;
        }
        cudaEventRecord(e1, b->st);
        cudaEventSynchronize(e1);
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        *ms = (double)x / steps;
        *span = sp > 0.0 ? sp : *ms;
        return rc;
    };
    double best_ms = 1e300;
    Cand bestc = shapes[0];
    int rc = PIC_OK;
    for (const Cand& c : shapes) {
        int r = batch_configure(b, c.block, c.bps, c.power, c.copies);
        if (r == PIC_ERR_UNSUPPORTED) continue;  // shape does not fit this batch
        if (r) {
            rc = r;
            break;
        }
        double ms = 0.0, span = 0.0;
        if ((rc = trial(steps_per_trial, &ms, &span))) break;
        if (span < best_ms) {
            best_ms = span;
            bestc = c;
        }
    }
    if (!rc) rc = batch_configure(b, bestc.block, bestc.bps, bestc.power, bestc.copies);
    // sort periods: whole periods are timed (at least steps_per_trial steps),
    // so that every trial holds one sort per period
    int best_sort = b->sort_every;
    if (!rc) {
        double best_sort_ms = 1e300;
        const int sorts[] = {1, 4, 16};
        for (int so : sorts) {
            b->sort_every = so;
            double ms = 0.0, span = 0.0;
            if ((rc = trial((steps_per_trial + so - 1) / so * so, &ms, &span))) break;
            if (ms < best_sort_ms) {
                best_sort_ms = ms;
                best_sort = so;
            }
        }
        b->sort_every = best_sort;
    }
    // Block shares from measured beam times (shares_minmax): the windows of
    // the last trial predict each beam's window on other block counts, and
    // the shares that minimise the largest prediction are tried next.  Up to
    // eight rounds, ended by two in a row that do not beat the best launch
    // span by 0.5 % (a slower trial still measures its own shares, so the
    // next round predicts from it); the shares that timed best stay.
    if (!rc) {
        double best_sh_ms = 0.0, ms0 = 0.0;
        rc = trial(steps_per_trial, &ms0, &best_sh_ms);
        BeamTimes best_t;  // empty: the power-law shares
        int misses = 0;
        for (int it = 0; it < 8 && !rc && misses < 2; ++it) {
            BeamTimes t;
            t.block = b->block;
            t.ms = beam_ms;
            t.blocks.resize(b->n);
            for (int i = 0; i < b->n; ++i) t.blocks[i] = b->desc[i].n_blocks;
            const int r = batch_configure(b, bestc.block, bestc.bps, bestc.power, bestc.copies, &t);
            if (r == PIC_ERR_UNSUPPORTED) break;
            if ((rc = r)) break;
            double ms = 0.0, span = 0.0;
            if ((rc = trial(steps_per_trial, &ms, &span))) break;
            if (span < 0.995 * best_sh_ms) {
                best_sh_ms = span;
                best_t = t;
                misses = 0;
            } else {
                ++misses;
            }
        }
        if (!rc)
            rc = batch_configure(b, bestc.block, bestc.bps, bestc.power, bestc.copies,
                                 best_t.ms.empty() ? nullptr : &best_t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return pic_batch_get_config(b, best);
}

int pic_test_batch_shares(int32_t n_beams, const int32_t* poisson, const int64_t* n_particles, const double* window_ms,
                          const int64_t* blocks_measured, int32_t block_measured, int32_t block, int64_t grid,
                          const int64_t* least, const int64_t* most, int64_t* blocks_out) {
    // bounds that keep blocks x threads + particles inside int64
    if (n_beams < 1 || !poisson || !n_particles || !window_ms || !blocks_measured || !least || !most || !blocks_out ||
        block_measured < 1 || block < 1 || block_measured > (1 << 20) || block > (1 << 20) || grid < 1 ||
        grid > (1ll << 31))
        return PIC_ERR_INVALID_ARG;
    const int n = n_beams;
    std::vector<char> coop(n);
    std::vector<long long> np(n), bm(n), lo(n), need(n), nb(n);
    std::vector<double> ms(n);
    for (int i = 0; i < n; ++i) {
        if (n_particles[i] < 1 || n_particles[i] > (1ll << 62) || blocks_measured[i] < 1 ||
            blocks_measured[i] > (1ll << 31) || least[i] < 1 || most[i] < least[i] || most[i] > (1ll << 31) ||
            !(window_ms[i] >= 0.0) || !std::isfinite(window_ms[i]))
            return PIC_ERR_INVALID_ARG;
        coop[i] = poisson[i] != 0;
        np[i] = n_particles[i];
        bm[i] = blocks_measured[i];
        lo[i] = least[i];
        need[i] = most[i];
        ms[i] = window_ms[i];
    }
    if (!shares_minmax_core(n, coop.data(), np.data(), ms.data(), bm.data(), block_measured, block, grid, lo.data(),
                            need.data(), nb.data()))
        return PIC_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) blocks_out[i] = nb[i];
    return PIC_OK;
}

int pic_batch_get_particles(pic_batch* b, int32_t beam, double* r, double* v, int ptr_kind) {
    if (!b || beam < 0 || beam >= b->n) return PIC_ERR_INVALID_ARG;
    return pic_get_particles(b->hs[beam], r, v, ptr_kind);
}

int pic_batch_set_particles(pic_batch* b, int32_t beam, const double* r, const double* v, int ptr_kind) {
    if (!b || beam < 0 || beam >= b->n) return PIC_ERR_INVALID_ARG;
    return pic_set_particles(b->hs[beam], r, v, ptr_kind);
}

int pic_batch_moments(pic_batch* b, int32_t beam, pic_moments_t* out) {
    if (!b || beam < 0 || beam >= b->n) return PIC_ERR_INVALID_ARG;
    return pic_moments(b->hs[beam], out);
}

int64_t pic_batch_steps(const pic_batch* b) { return b ? b->steps : -1; }

int64_t pic_batch_launch_count(const pic_batch* b) { return b ? b->launches : -1; }

void pic_batch_destroy(pic_batch* b) { batch_free(b); }

}  // extern "C"

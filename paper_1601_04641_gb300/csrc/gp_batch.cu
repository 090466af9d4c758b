// gp_batch.cu -- many independent condensates (uneven grids, traps and g)
// advanced together: every imaginary-time step is one launch per sweep
// (kick + x, y, z + norm) over all active instances -- two on a strided axis
// when some instances advance line pairs and others single lines -- with
// per-instance argument blocks, norm partials and completion counters;
// blocks of steps are replayed from captured CUDA graphs; converged
// instances drop out of the launches.
#include "gp.h"
#include "gp_host.h"
#include "gp_internal.h"
#include "gp_nn_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

using namespace gpcn;

namespace {

struct Inst {
    Geometry G;
    double dt0 = 0.0;       // the step given at creation (G.dt = dt0 * the batch's dt scale)
    Tables tab;
    size_t psi_off = 0;     // byte offset in each packed psi buffer
    size_t sites = 0, bytes = 0;
    size_t part_off = 0;    // offset (doubles) of the partials region
    int seg_len[3] = {0, 0, 0}, n_seg[3] = {0, 0, 0};
    int lpt[3] = {1, 1, 1}; // lines per thread of the strided sweeps (2: adjacent line pairs)
    bool ztma = false;      // z sweep through TMA tiles (its rows fit the TMA form)
    int cur = 0;            // which packed buffer holds psi
    long long step = 0;
    double t = 0.0;
    bool active = true;
};

// Device tables of one launch configuration (a set of instances, a parity).
// Each sweep has up to two launches.  Strided sweeps: group 0 the instances
// that advance one line per thread, group 1 those that advance adjacent line
// pairs.  z sweep: group 0 the per-thread-copy form, group 1 the TMA form
// (at most kTmaBatch instances whose rows fit it, with their tensor maps).
struct SweepSet {
    SweepArgs *args[3][2][2] = {};   // [sweep][group][parity]
    unsigned *first[3][2] = {};
    unsigned *gridx[3][2] = {};
    unsigned total[3][2] = {};
    int count[3][2] = {};
    std::vector<BatchTmaMaps> zmaps;  // [parity]: maps of the z sweep's TMA group
};

// The active instances, split into stream groups: each group's x, y and z
// sweeps form one chain of launches on its own stream (the groups'
// condensates are independent), so the launches of different groups overlap
// and fill each other's ramp-up and tail.
struct LaunchSet {
    std::vector<SweepSet> sets;   // one per stream group
    FieldArgs *fargs = nullptr;   // observables of the instances, for their current parity
    unsigned *ofirst = nullptr;
    unsigned ototal = 0;
    std::vector<int> members;
    int parity = 0;               // steps taken by the members since the tables were built, mod 2
};

constexpr int kSweepThreads = kBatchLineThreads;  // both batched sweep kernels use 64 threads
constexpr int kInitNormBlocks = 152 * 4;

}  // namespace

struct gp_batch_s {
    int device = 0;
    int n = 0;
    gp_precision prec = GP_F32;
    gp_field field = GP_COMPLEX;
    size_t elem = 0;
    cudaStream_t stream = nullptr;
    std::vector<Inst> inst;
    char *d_psi[2] = {nullptr, nullptr};
    size_t psi_bytes = 0;
    char *d_tab = nullptr;
    double *d_scal = nullptr;      // per instance: [scale, norm]
    double *d_obs = nullptr;       // per instance: O_COUNT values
    double *d_partials = nullptr;
    unsigned int *d_counters = nullptr;
    int window[3] = {0, 0, 0};
    bool contiguous_z = false;
    bool use_tma = true;           // z sweep through TMA for the instances whose rows fit
    int seg_len = 0;               // interior nodes per segment on the strided axes (0: automatic)
    LaunchSet act;                 // the active instances
    int streams = 2;               // stream groups of a step (1: one chain of launches)
    std::vector<cudaStream_t> gstream;   // the groups' streams (created on first use)
    std::vector<cudaEvent_t> gevent;     // fork event, then one join event per group
    bool dirty = true;
    int graph_block = 16;
    int stop_rule = 0;             // as gp_set_stop_rule (0, 1 or 2)
    double dt_scale = 1.0;         // every instance steps with dt0 * dt_scale
    size_t tab_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (parity, steps)
    std::vector<void *> scratch;   // device allocations of the launch sets
    std::string err;
};

namespace {

gp_status bfail(gp_batch b, gp_status st, const std::string &m) {
    if (b) b->err = m;
    else set_thread_error(m.c_str());
    return st;
}

#define GPB_CK(b, call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bfail((b), GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

void free_set(gp_batch b) {
    for (void *p : b->scratch) cudaFree(p);
    b->scratch.clear();
    b->act = LaunchSet();
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <typename T> gp_status upload(gp_batch b, const std::vector<T> &v, T **out) {
    *out = nullptr;
    if (v.empty()) return GP_OK;
    void *p = nullptr;
    if (gpcn::dev_malloc(&p, v.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, GP_ERR_NOMEM, "cudaMalloc of batch launch tables failed");
    }
    b->scratch.push_back(p);
    GPB_CK(b, cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream));
    *out = static_cast<T *>(p);
    return GP_OK;
}

unsigned sweep_gridx(gp_batch b, const Inst &I, int ax, int lpt = 1) {
    const long long units = (axis_lines(I.G, ax) + lpt - 1) / lpt;
    (void)b;
    return (unsigned)((units + kSweepThreads - 1) / kSweepThreads);
}

// Which instances take the TMA z sweep: the first kTmaBatch whose rows fit
// the TMA form at the batch's z window (the contiguous z sweep solves whole
// lines, one segment).
void assign_ztma(gp_batch b) {
    int count = 0;
    for (Inst &I : b->inst) {
        I.ztma = b->use_tma && b->contiguous_z && count < kTmaBatch &&
                 tma_z_fits((int)b->elem, b->window[2], I.G.n[2], 1, axis_lines(I.G, 2));
        count += I.ztma ? 1 : 0;
    }
}

void assign_segments(gp_batch b);

// Tables, windows and segments of every instance for dt = dt0 * scale.  One
// window per axis for the whole batch: the largest of the instances' smallest
// admissible windows (0 if any instance admits none, or FP64).
void configure(gp_batch b, double scale, std::vector<char> &host) {
    const bool f32 = b->prec == GP_F32;
    host.clear();
    for (Inst &I : b->inst) {
        I.G.dt = I.dt0 * scale;
        I.tab = Tables();
        append_tables(I.G, f32, 1, host, I.tab);
    }
    for (int ax = 0; ax < 3; ++ax) {
        int w = 0;
        bool all = f32;
        for (size_t i = 0; i < b->inst.size() && all; ++i) {
            const int m = b->inst[i].tab.ax[0][ax].min_window;
            if (m == 0) all = false;
            w = std::max(w, m);
        }
        b->window[ax] = all ? w : 0;
    }
    b->contiguous_z = b->window[2] > 0;
    assign_ztma(b);
    assign_segments(b);
    b->dt_scale = scale;
}

// Lines per thread and segments of every instance and axis at the batch's
// windows (segment length override b->seg_len on the strided axes).
void assign_segments(gp_batch b) {
    for (Inst &I : b->inst)
        for (int ax = 0; ax < 3; ++ax) {
            // adjacent line pairs on a strided axis (window 4, 8-byte
            // elements) when every pair is adjacent in memory: an even number
            // of lines and, for y lines (i, k), an even nz.  Measured on the
            // 64-condensate workload: complex64 0.312 -> 0.298 ms per step;
            // FP32 real fields (8 bytes per pair node) 0.196 -> 0.208, as
            // pairing halves the threads of these small grids.  A pair cuts
            // lines into 8-node chunks, each re-running W back steps: at
            // windows 8 and 16 (the coarse levels of a dt schedule) that
            // overhead outweighs the packed arithmetic (schedule 0.451 ->
            // 0.479 s with pairs at every window)
            const bool pair = ax < 2 && b->window[ax] == 4 && b->elem == 8 && axis_lines(I.G, ax) % 2 == 0 &&
                              (ax != 1 || I.G.n[2] % 2 == 0);
            I.lpt[ax] = pair ? 2 : 1;
            choose_segments(I.G, ax, b->window[ax], I.lpt[ax], (int)b->elem, ax == 2 && b->contiguous_z,
                            ax < 2 ? b->seg_len : 0, &I.seg_len[ax], &I.n_seg[ax]);
        }
}

// Norm / observables partials an instance may need under any window choice
// (the windowed forms cut the strided axes into the most segments).
size_t partial_cap(gp_batch b, const Inst &I) {
    size_t cap = kInitNormBlocks;
    for (int ax = 0; ax < 3; ++ax) {
        int len, nseg;
        choose_segments(I.G, ax, 4, 1, (int)b->elem, ax == 2, 0, &len, &nseg);
        cap = std::max(cap, (size_t)sweep_gridx(b, I, ax) * nseg);
        choose_segments(I.G, ax, 0, 1, (int)b->elem, false, 0, &len, &nseg);
        cap = std::max(cap, (size_t)sweep_gridx(b, I, ax) * nseg);
    }
    FieldArgs fa = field_args(I.G, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return std::max(cap, (size_t)observables_blocks(fa) * 9);
}

FieldArgs inst_field_args(gp_batch b, int i) {
    const Inst &I = b->inst[i];
    return field_args(I.G, b->d_psi[I.cur] + I.psi_off, b->d_scal + 2 * i, b->d_partials + I.part_off,
                      b->d_counters + i, b->d_obs + (size_t)i * O_COUNT, b->d_scal + 2 * i,
                      b->d_scal + 2 * i + 1);
}

// Device tables for the active instances at their current parity.
gp_status build_set(gp_batch b) {
    free_set(b);
    LaunchSet &S = b->act;
    for (int i = 0; i < b->n; ++i)
        if (b->inst[i].active) S.members.push_back(i);
    // stream groups balanced by sites: largest instance first to the least
    // loaded group
    const int ng = std::max(1, std::min(b->streams, (int)S.members.size()));
    std::vector<std::vector<int>> groups(ng);
    {
        std::vector<int> bysize(S.members);
        std::stable_sort(bysize.begin(), bysize.end(),
                         [&](int a, int c) { return b->inst[a].sites > b->inst[c].sites; });
        std::vector<size_t> load(ng, 0);
        for (int i : bysize) {
            const int gi = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            groups[gi].push_back(i);
            load[gi] += b->inst[i].sites;
        }
    }
    S.sets.assign(ng, SweepSet());
    for (int gs = 0; gs < ng; ++gs) {
        SweepSet &T = S.sets[gs];
        T.zmaps.assign(2, BatchTmaMaps());
        for (int k = 0; k < 3; ++k) {
            // longest lines first: a block's run time grows with its lines'
            // length, and blocks start in grid order, so the long ones should
            // not be left for the end of the launch (instances are independent;
            // their order changes no result)
            std::vector<int> order(groups[gs]);
            std::stable_sort(order.begin(), order.end(),
                             [&](int a, int c) { return b->inst[a].G.n[k] > b->inst[c].G.n[k]; });
            for (int g = 0; g < 2; ++g) {
                std::vector<SweepArgs> args[2];
                std::vector<unsigned> first{0}, gridx;
                for (int i : order) {
                    const Inst &I = b->inst[i];
                    const bool tma = k == 2 && I.ztma;
                    if (k == 2 ? (tma != (g == 1)) : I.lpt[k] != g + 1) continue;
                    for (int p = 0; p < 2; ++p) {
                        // sweep k of a step that starts with psi in buffer I.cur ^ p
                        const int in = I.cur ^ p ^ (k & 1);
                        const char *src = b->d_psi[in] + I.psi_off;
                        char *dst = b->d_psi[in ^ 1] + I.psi_off;
                        args[p].push_back(sweep_args(I.G, k, false, src, dst, b->d_tab, I.tab, I.seg_len[k],
                                                     I.n_seg[k], b->d_scal + 2 * i, b->d_partials + I.part_off,
                                                     b->d_counters + i, b->d_scal + 2 * i + 1, b->d_scal + 2 * i));
                        if (tma) {
                            const size_t q = args[p].size() - 1;
                            const long long rows = axis_lines(I.G, 2);
                            if (!encode_z_map(&T.zmaps[p].in[q], src, I.G.n[2], rows, (int)b->elem) ||
                                !encode_z_map(&T.zmaps[p].out[q], dst, I.G.n[2], rows, (int)b->elem))
                                return bfail(b, GP_ERR_CUDA, "encoding a tensor map of the batched z sweep failed");
                        }
                    }
                    // TMA: one block per kTmaWarps * 64 rows, as a single-condensate launch
                    const unsigned gx = tma ? (unsigned)((axis_lines(I.G, 2) + kTmaBlockRows - 1) / kTmaBlockRows)
                                            : sweep_gridx(b, I, k, I.lpt[k]);
                    gridx.push_back(gx);
                    first.push_back(first.back() + gx * (unsigned)I.n_seg[k]);
                }
                T.total[k][g] = first.back();
                T.count[k][g] = (int)gridx.size();
                gp_status st;
                if ((st = upload(b, args[0], &T.args[k][g][0])) != GP_OK) return st;
                if ((st = upload(b, args[1], &T.args[k][g][1])) != GP_OK) return st;
                if ((st = upload(b, first, &T.first[k][g])) != GP_OK) return st;
                if ((st = upload(b, gridx, &T.gridx[k][g])) != GP_OK) return st;
            }
        }
    }
    // the groups' streams and events, made here, outside any stream capture
    while ((int)b->gstream.size() < ng && ng > 1) {
        cudaStream_t gs = nullptr;
        GPB_CK(b, cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
        b->gstream.push_back(gs);
    }
    while ((int)b->gevent.size() < ng + 1 && ng > 1) {
        cudaEvent_t e = nullptr;
        GPB_CK(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->gevent.push_back(e);
    }
    std::vector<FieldArgs> fa;
    std::vector<unsigned> of{0};
    for (int i : S.members) {
        fa.push_back(inst_field_args(b, i));
        of.push_back(of.back() + (unsigned)observables_body_blocks(fa.back()));
    }
    S.ototal = of.back();
    gp_status st;
    if ((st = upload(b, fa, &S.fargs)) != GP_OK) return st;
    if ((st = upload(b, of, &S.ofirst)) != GP_OK) return st;
    S.parity = 0;
    b->dirty = false;
    return GP_OK;
}

gp_status launch_sweeps(gp_batch b, const SweepSet &T, cudaStream_t s, int parity) {
    for (int k = 0; k < 3; ++k) {
        SweepLaunch L;
        L.prec = b->prec == GP_F32 ? P_F32 : P_F64;
        L.form = b->field == GP_REAL ? F_IMAG_REAL : F_IMAG_CPLX;
        L.kind = static_cast<Kind>(k);
        L.window = b->window[k];
        L.threads = kSweepThreads;
        L.contiguous = (k == 2 && b->contiguous_z) ? 1 : 0;
        for (int g = 0; g < 2; ++g) {
            if (T.count[k][g] == 0) continue;
            L.lpt = k < 2 ? g + 1 : 1;
            BatchLaunch bl{T.args[k][g][parity], T.first[k][g], T.gridx[k][g], T.count[k][g], T.total[k][g]};
            if (k == 2 && g == 1) bl.tma = &T.zmaps[parity];
            GPB_CK(b, launch_sweep_batch(L, bl, s));
        }
    }
    return GP_OK;
}

// One step of the active instances queued on s: with one stream group, the
// sweeps on s; with several, each group's sweeps on its own stream, forked
// from and joined back into s by events (a capture on s records the groups
// as parallel branches of the graph).
gp_status launch_step(gp_batch b, cudaStream_t s, int parity) {
    LaunchSet &S = b->act;
    const int ng = (int)S.sets.size();
    if (ng == 1) return launch_sweeps(b, S.sets[0], s, parity);
    if ((int)b->gstream.size() < ng || (int)b->gevent.size() < ng + 1)
        return bfail(b, GP_ERR_STATE, "stream groups not set up");
    GPB_CK(b, cudaEventRecord(b->gevent[0], s));
    for (int g = 0; g < ng; ++g) {
        GPB_CK(b, cudaStreamWaitEvent(b->gstream[g], b->gevent[0], 0));
        gp_status st = launch_sweeps(b, S.sets[g], b->gstream[g], parity);
        if (st != GP_OK) return st;
        GPB_CK(b, cudaEventRecord(b->gevent[g + 1], b->gstream[g]));
        GPB_CK(b, cudaStreamWaitEvent(s, b->gevent[g + 1], 0));
    }
    return GP_OK;
}

// After n steps of the active instances.
void advance(gp_batch b, int n) {
    for (int i : b->act.members) {
        Inst &I = b->inst[i];
        if (n % 2) I.cur ^= 1;  // three sweeps per step
        I.step += n;
        for (int k = 0; k < n; ++k) I.t += I.G.dt;
    }
    b->act.parity = (b->act.parity + n) & 1;
}

gp_status run_graph(gp_batch b, int g) {
    const auto key = std::make_pair(b->act.parity, g);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        gp_status st = GP_OK;
        for (int s = 0; s < g && st == GP_OK; ++s) st = launch_step(b, b->cap_stream, (b->act.parity + s) & 1);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        const bool ok = st == GP_OK && ec == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        it = b->graphs.emplace(key, exec).first;
    }
    GPB_CK(b, cudaGraphLaunch(it->second, b->stream));
    return GP_OK;
}

gp_status step_active(gp_batch b, int nsteps) {
    if (b->dirty) {
        gp_status st = build_set(b);
        if (st != GP_OK) return st;
    }
    if (b->act.members.empty()) return GP_OK;
    while (nsteps > 0) {
        const int g = std::min(nsteps, std::max(1, b->graph_block));
        gp_status st = GP_ERR_STATE;
        if (g > 1) st = run_graph(b, g);
        if (st == GP_ERR_STATE) {
            for (int s = 0; s < g; ++s) {
                st = launch_step(b, b->stream, (b->act.parity + s) & 1);
                if (st != GP_OK) return st;
            }
        } else if (st != GP_OK) {
            return st;
        }
        advance(b, g);
        nsteps -= g;
    }
    return GP_OK;
}

// Observables of the active instances into host memory (one record per instance).
gp_status observe_active(gp_batch b, std::vector<double> &host) {
    LaunchSet &S = b->act;
    if (S.members.empty()) return GP_OK;
    // the field arguments follow each instance's current buffer
    std::vector<FieldArgs> fa;
    for (int i : S.members) fa.push_back(inst_field_args(b, i));
    GPB_CK(b, cudaMemcpyAsync(S.fargs, fa.data(), fa.size() * sizeof(FieldArgs), cudaMemcpyHostToDevice, b->stream));
    GPB_CK(b, launch_observables_batch(b->prec == GP_F32 ? P_F32 : P_F64, b->field == GP_COMPLEX, S.fargs, S.ofirst,
                                       (int)S.members.size(), S.ototal, b->stream));
    host.assign((size_t)b->n * O_COUNT, 0.0);
    GPB_CK(b, cudaMemcpyAsync(host.data(), b->d_obs, host.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    return GP_OK;
}

void release_batch(gp_batch b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_set(b);
    cudaFree(b->d_psi[0]);
    cudaFree(b->d_psi[1]);
    cudaFree(b->d_tab);
    cudaFree(b->d_scal);
    cudaFree(b->d_obs);
    cudaFree(b->d_partials);
    cudaFree(b->d_counters);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaStream_t gs : b->gstream) cudaStreamDestroy(gs);
    for (cudaEvent_t e : b->gevent) cudaEventDestroy(e);
    cudaGetLastError();
    delete b;
}

gp_status benter(gp_batch b) {
    if (!b) return bfail(nullptr, GP_ERR_ARG, "NULL batch");
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, GP_ERR_CUDA, "cudaSetDevice failed");
    }
    return GP_OK;
}

void fill_obs(const double *o, const Inst &I, gp_obs *out) {
    out->norm = o[O_NORM];
    out->mu = o[O_MU];
    out->energy = o[O_E];
    out->rms_x = o[O_RMSX];
    out->rms_y = o[O_RMSY];
    out->rms_z = o[O_RMSZ];
    out->step = I.step;
    out->t = I.t;
}

}  // namespace

extern "C" {

gp_status gp_batch_create(gp_batch *out, int n, const gp_grid *grids, const double *dt, const double *gamma,
                          const double *nu, const double *lambda, const double *g, gp_precision prec,
                          gp_field field, void *cuda_stream) {
    if (!out) return bfail(nullptr, GP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !dt || !gamma || !nu || !lambda || !g)
        return bfail(nullptr, GP_ERR_ARG, "need n >= 1 and all parameter arrays");
    if (prec == GP_F16) return bfail(nullptr, GP_ERR_ARG, "the batched form has no FP16 storage");
    if (prec != GP_F64 && prec != GP_F32) return bfail(nullptr, GP_ERR_ARG, "unknown precision");
    if (field != GP_COMPLEX && field != GP_REAL) return bfail(nullptr, GP_ERR_ARG, "unknown field");
    for (int i = 0; i < n; ++i) {
        const int nn[3] = {grids[i].nx, grids[i].ny, grids[i].nz};
        const double dd[3] = {grids[i].dx, grids[i].dy, grids[i].dz};
        for (int a = 0; a < 3; ++a)
            if (nn[a] < 3 || !(dd[a] > 0.0) || !std::isfinite(dd[a]))
                return bfail(nullptr, GP_ERR_ARG, "instance " + std::to_string(i) + ": bad grid");
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i]) || !std::isfinite(g[i]))
            return bfail(nullptr, GP_ERR_ARG, "instance " + std::to_string(i) + ": bad dt or g");
        const double w[3] = {gamma[i], nu[i], lambda[i]};
        for (double x : w)
            if (!std::isfinite(x) || x < 0.0)
                return bfail(nullptr, GP_ERR_ARG, "instance " + std::to_string(i) + ": bad trap frequency");
    }
    gp_batch b = new (std::nothrow) gp_batch_s();
    if (!b) return bfail(nullptr, GP_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(nullptr, GP_ERR_CUDA, "no CUDA device");
    }
    prepare_field_launches();
    b->n = n;
    b->prec = prec;
    b->field = field;
    b->elem = (prec == GP_F64 ? 8 : 4) * (field == GP_COMPLEX ? 2 : 1);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->inst.resize(n);
    std::vector<char> host;
    size_t psi = 0, parts = 0;
    for (int i = 0; i < n; ++i) {
        Inst &I = b->inst[i];
        I.G.n[0] = grids[i].nx;
        I.G.n[1] = grids[i].ny;
        I.G.n[2] = grids[i].nz;
        I.G.d[0] = grids[i].dx;
        I.G.d[1] = grids[i].dy;
        I.G.d[2] = grids[i].dz;
        I.dt0 = dt[i];
        I.G.w[0] = gamma[i];
        I.G.w[1] = nu[i];
        I.G.w[2] = lambda[i];
        I.G.g = g[i];
        I.sites = (size_t)grids[i].nx * grids[i].ny * grids[i].nz;
        I.bytes = I.sites * b->elem;
        I.psi_off = psi;
        psi = align_up(psi + I.bytes, 256);
    }
    configure(b, 1.0, host);
    for (int i = 0; i < n; ++i) {
        Inst &I = b->inst[i];
        I.part_off = parts;
        parts += align_up(partial_cap(b, I), 32);
    }
    b->psi_bytes = psi;
    b->tab_bytes = host.size();
    if (gpcn::dev_malloc(&b->d_psi[0], psi) != cudaSuccess || gpcn::dev_malloc(&b->d_psi[1], psi) != cudaSuccess ||
        gpcn::dev_malloc(&b->d_tab, host.size()) != cudaSuccess ||
        gpcn::dev_malloc(&b->d_scal, 2 * n * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&b->d_obs, (size_t)n * O_COUNT * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&b->d_partials, parts * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&b->d_counters, n * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        release_batch(b);
        return bfail(nullptr, GP_ERR_NOMEM, "device allocation of the batch failed");
    }
    std::vector<double> scal(2 * n, 1.0);
    if (cudaMemcpyAsync(b->d_tab, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_scal, scal.data(), scal.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->d_counters, 0, n * sizeof(unsigned int), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_psi[0], 0, psi, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        release_batch(b);
        return bfail(nullptr, GP_ERR_CUDA, "initialising the batch failed");
    }
    *out = b;
    return GP_OK;
}

void gp_batch_destroy(gp_batch b) { release_batch(b); }

gp_status gp_batch_init_gaussian(gp_batch b) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    const Prec p = b->prec == GP_F32 ? P_F32 : P_F64;
    const bool cplx = b->field == GP_COMPLEX;
    for (int i = 0; i < b->n; ++i) {
        FieldArgs a = inst_field_args(b, i);
        GPB_CK(b, launch_gaussian(p, cplx, a, b->stream));
        GPB_CK(b, launch_norm(p, cplx, a, kInitNormBlocks, b->stream));
        b->inst[i].step = 0;
        b->inst[i].t = 0.0;
    }
    b->dirty = true;
    return GP_OK;
}

gp_status gp_batch_set_psi(gp_batch b, int i, const void *psi, int on_device) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (i < 0 || i >= b->n || !psi) return bfail(b, GP_ERR_ARG, "bad instance or NULL psi");
    Inst &I = b->inst[i];
    GPB_CK(b, cudaMemcpyAsync(b->d_psi[I.cur] + I.psi_off, psi, I.bytes,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    const double one = 1.0;
    GPB_CK(b, cudaMemcpyAsync(b->d_scal + 2 * i, &one, sizeof(one), cudaMemcpyHostToDevice, b->stream));
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    I.step = 0;
    I.t = 0.0;
    return GP_OK;
}

gp_status gp_batch_get_psi(gp_batch b, int i, void *psi, int on_device) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (i < 0 || i >= b->n || !psi) return bfail(b, GP_ERR_ARG, "bad instance or NULL psi");
    Inst &I = b->inst[i];
    FieldArgs a = inst_field_args(b, i);
    const Prec p = b->prec == GP_F32 ? P_F32 : P_F64;
    const bool cplx = b->field == GP_COMPLEX;
    if (on_device) {
        GPB_CK(b, launch_apply_scale(p, cplx, a, psi, b->stream));
        return GP_OK;
    }
    // apply the pending factor into the other buffer, copy it out
    char *tmp = b->d_psi[I.cur ^ 1] + I.psi_off;
    GPB_CK(b, launch_apply_scale(p, cplx, a, tmp, b->stream));
    GPB_CK(b, cudaMemcpyAsync(psi, tmp, I.bytes, cudaMemcpyDeviceToHost, b->stream));
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    return GP_OK;
}

gp_status gp_batch_step_imag(gp_batch b, int nsteps) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (nsteps < 0) return bfail(b, GP_ERR_ARG, "nsteps < 0");
    return step_active(b, nsteps);
}

gp_status gp_batch_observables(gp_batch b, gp_obs *out) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (!out) return bfail(b, GP_ERR_ARG, "out is NULL");
    const Prec p = b->prec == GP_F32 ? P_F32 : P_F64;
    const bool cplx = b->field == GP_COMPLEX;
    for (int i = 0; i < b->n; ++i) {
        FieldArgs a = inst_field_args(b, i);
        GPB_CK(b, launch_observables(p, cplx, a, b->stream));
    }
    std::vector<double> host((size_t)b->n * O_COUNT);
    GPB_CK(b, cudaMemcpyAsync(host.data(), b->d_obs, host.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    bool finite = true;
    for (int i = 0; i < b->n; ++i) {
        fill_obs(host.data() + (size_t)i * O_COUNT, b->inst[i], out + i);
        finite = finite && host[(size_t)i * O_COUNT + O_FINITE] == 1.0;
    }
    if (!finite) return bfail(b, GP_ERR_NONFINITE, "an instance's psi holds NaN or Inf");
    return GP_OK;
}

gp_status gp_batch_run_imag_until(gp_batch b, double mu_tol, int check_every, int max_steps, int *steps_taken) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (!(mu_tol > 0.0) || check_every < 1 || max_steps < 0)
        return bfail(b, GP_ERR_ARG, "need mu_tol > 0, check_every >= 1, max_steps >= 0");
    for (int i = 0; i < b->n; ++i) b->inst[i].active = true;
    b->dirty = true;
    if ((st = build_set(b)) != GP_OK) return st;
    std::vector<double> host;
    if ((st = observe_active(b, host)) != GP_OK) return st;
    std::vector<double> mu_prev(b->n), e_prev(b->n);
    std::vector<int> taken(b->n, 0), streak(b->n, 0);
    const int need = b->stop_rule == 2 ? 2 : 1;  // consecutive checks that must pass
    for (int i = 0; i < b->n; ++i) {
        mu_prev[i] = host[(size_t)i * O_COUNT + O_MU];
        e_prev[i] = host[(size_t)i * O_COUNT + O_E];
    }
    int done = 0;
    while (done < max_steps && !b->act.members.empty()) {
        const int n = std::min(check_every, max_steps - done);
        if ((st = step_active(b, n)) != GP_OK) break;
        done += n;
        if ((st = observe_active(b, host)) != GP_OK) break;
        bool changed = false;
        for (int i : b->act.members) {
            const double *o = host.data() + (size_t)i * O_COUNT;
            taken[i] = done;
            if (o[O_FINITE] != 1.0) {
                st = bfail(b, GP_ERR_NONFINITE, "instance " + std::to_string(i) + " became non-finite");
                break;
            }
            const bool pass = std::fabs(o[O_MU] - mu_prev[i]) < mu_tol &&
                              (b->stop_rule == 0 || std::fabs(o[O_E] - e_prev[i]) < mu_tol);
            streak[i] = pass ? streak[i] + 1 : 0;
            if (streak[i] >= need) {
                b->inst[i].active = false;
                changed = true;
            }
            mu_prev[i] = o[O_MU];
            e_prev[i] = o[O_E];
        }
        if (st != GP_OK) break;
        if (changed) {
            b->dirty = true;
            if ((st = build_set(b)) != GP_OK) break;
        }
    }
    if (steps_taken)
        for (int i = 0; i < b->n; ++i) steps_taken[i] = taken[i];
    for (int i = 0; i < b->n; ++i) b->inst[i].active = true;
    b->dirty = true;
    return st;
}

gp_status gp_batch_get_window(gp_batch b, int window[3]) {
    if (!b || !window) return bfail(b, GP_ERR_ARG, "bad arguments");
    for (int ax = 0; ax < 3; ++ax) window[ax] = b->window[ax];
    return GP_OK;
}

gp_status gp_batch_get_segments(gp_batch b, int i, int seg_len[3], int n_seg[3]) {
    if (!b || !seg_len || !n_seg || i < 0 || i >= b->n) return bfail(b, GP_ERR_ARG, "bad arguments");
    for (int ax = 0; ax < 3; ++ax) {
        seg_len[ax] = b->inst[i].seg_len[ax];
        n_seg[ax] = b->inst[i].n_seg[ax];
    }
    return GP_OK;
}

gp_status gp_nn_predict_batch(gp_nn net, gp_batch b) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    const NNParams *P = nn_params(net);
    if (!P) return bfail(b, GP_ERR_ARG, "NULL network");
    const Prec p = b->prec == GP_F32 ? P_F32 : P_F64;
    const bool cplx = b->field == GP_COMPLEX;
    for (int i = 0; i < b->n; ++i) {
        Inst &I = b->inst[i];
        const NNInstance ni = make_nn_instance(I.G.n, I.G.d, I.G.w, I.G.g);
        GPB_CK(b, nn_launch_predict(*P, ni, b->d_psi[I.cur] + I.psi_off, b->prec == GP_F32, cplx, b->stream));
        FieldArgs a = inst_field_args(b, i);
        GPB_CK(b, launch_norm(p, cplx, a, kInitNormBlocks, b->stream));
        I.step = 0;
        I.t = 0.0;
    }
    return GP_OK;
}

gp_status gp_batch_set_dt_scale(gp_batch b, double scale) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (!(scale > 0.0) || !std::isfinite(scale)) return bfail(b, GP_ERR_ARG, "scale must be finite and > 0");
    if (scale == b->dt_scale) return GP_OK;
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    std::vector<char> host;
    configure(b, scale, host);
    if (host.size() != b->tab_bytes) return bfail(b, GP_ERR_STATE, "table layout changed with dt");
    GPB_CK(b, cudaMemcpyAsync(b->d_tab, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream));
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    free_set(b);
    b->dirty = true;
    return GP_OK;
}

gp_status gp_batch_run_imag_schedule(gp_batch b, int levels, const double *dt_scale, const double *mu_tol,
                                     int check_every, int max_steps, int *steps_taken) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (levels < 1 || !dt_scale || !mu_tol) return bfail(b, GP_ERR_ARG, "need levels >= 1 and both arrays");
    std::vector<int> total(b->n, 0), part(b->n, 0);
    const double base = b->dt_scale;
    for (int l = 0; l < levels && st == GP_OK; ++l) {
        st = gp_batch_set_dt_scale(b, base * dt_scale[l]);
        if (st == GP_OK) st = gp_batch_run_imag_until(b, mu_tol[l], check_every, max_steps, part.data());
        for (int i = 0; i < b->n; ++i) total[i] += part[i];
    }
    const gp_status back = gp_batch_set_dt_scale(b, base);
    if (st == GP_OK) st = back;
    if (steps_taken)
        for (int i = 0; i < b->n; ++i) steps_taken[i] = total[i];
    return st;
}

gp_status gp_batch_set_stop_rule(gp_batch b, int rule) {
    if (!b) return bfail(b, GP_ERR_ARG, "NULL batch");
    if (rule < 0 || rule > 2) return bfail(b, GP_ERR_ARG, "rule must be 0, 1 or 2");
    b->stop_rule = rule;
    return GP_OK;
}

gp_status gp_batch_set_tma(gp_batch b, int on) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    b->use_tma = on != 0;
    assign_ztma(b);
    free_set(b);
    b->dirty = true;
    return GP_OK;
}

gp_status gp_batch_set_streams(gp_batch b, int streams) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (streams < 1 || streams > 16) return bfail(b, GP_ERR_ARG, "streams must be in [1, 16]");
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    b->streams = streams;
    free_set(b);
    b->dirty = true;
    return GP_OK;
}

gp_status gp_batch_set_segments(gp_batch b, int seg_len) {
    gp_status st = benter(b);
    if (st != GP_OK) return st;
    if (seg_len < 0) return bfail(b, GP_ERR_ARG, "seg_len must be >= 0");
    GPB_CK(b, cudaStreamSynchronize(b->stream));
    b->seg_len = seg_len;
    assign_segments(b);
    free_set(b);
    b->dirty = true;
    return GP_OK;
}

gp_status gp_batch_get_tma(gp_batch b, int *count) {
    if (!b || !count) return bfail(b, GP_ERR_ARG, "bad arguments");
    int c = 0;
    for (const Inst &I : b->inst) c += I.ztma ? 1 : 0;
    *count = c;
    return GP_OK;
}

gp_status gp_batch_set_graph_block(gp_batch b, int steps) {
    if (!b) return bfail(b, GP_ERR_ARG, "NULL batch");
    if (steps < 0 || steps > 1024) return bfail(b, GP_ERR_ARG, "steps must be in [0, 1024]");
    b->graph_block = steps;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return GP_OK;
}

const char *gp_batch_last_error(gp_batch b) {
    if (!b) return gp_last_error(nullptr);
    return b->err.c_str();
}

}  // extern "C"

// Many separate problems of uneven size, each with its own AIRG hierarchy,
// solved together.  FGMRES runs in lockstep across the problems; iteration j
// of all of them is one CUDA graph launch, captured once per j, in which
// every problem forms an independent branch:
//     [scale v_j = w / ||w||] -> V-cycle(v_j -> z_j) -> w = A z_j
//     -> h = V^T w (with <w,w>) -> w -= V h, ||w||^2
// so the GPU runs the branches of small problems side by side.  One host
// synchronisation per iteration reads every problem's Hessenberg column;
// the rare second Gram-Schmidt pass and the restarts run as direct launches
// on per-problem streams.  A converged problem is frozen: its scale factor
// is zero and its least-squares solution uses the columns it built while
// active.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "dev_util.cuh"
#include "handle.h"
#include "solve_internal.cuh"
#include "worklist.h"

namespace airg {
void set_last_error(const char* msg);
DevCSR upload_csr_checked(const airg_csr* A, cudaStream_t st);
void check_options_checked(const airg_options& o);
}  // namespace airg

struct airg_batch_s {
    std::vector<std::unique_ptr<airg::Hierarchy>> H;
    std::vector<cudaStream_t> ps;      // one stream per problem
    cudaStream_t master = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<airg::DBuf<double>> dv;    // per problem: h1 | h2 | nrm | ww | bn | rn
    std::vector<airg::DBuf<int>> act;      // per problem: active flag read by the graph
    airg::HBuf<double> hbuf;               // pinned copies of every dv
    std::vector<cudaGraphExec_t> graphs;   // per iteration index j
    cudaGraphExec_t rich = nullptr;        // one Richardson iteration
    std::vector<std::vector<long long>> gk;   // kernels per problem in graphs[j]
    std::vector<long long> rk;                // kernels per problem in rich
    std::vector<airg::DBuf<double>> stage_b, stage_x;   // device copies of host b, x
    // persistent work-list form: one list and one captured launch per j
    std::vector<std::shared_ptr<airg::WorkList>> wls;
    std::vector<cudaGraphExec_t> wgraphs;
    // optional timing of the iteration launches (airg_batch_profile)
    bool prof = false;
    double prof_ms = 0.0;
    long long prof_launches = 0, prof_bytes = 0;
    cudaEvent_t pev[2] = {nullptr, nullptr};
    std::vector<std::vector<long long>> it_bytes;   // [j][p] algorithmic bytes of iteration j
    int m = 0;
    ~airg_batch_s()
    {
        for (cudaEvent_t e : pev)
            if (e) cudaEventDestroy(e);
        for (cudaGraphExec_t g : wgraphs)
            if (g) cudaGraphExecDestroy(g);
        for (cudaGraphExec_t g : graphs)
            if (g) cudaGraphExecDestroy(g);
        if (rich) cudaGraphExecDestroy(rich);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : ps) cudaStreamDestroy(s);
        if (master) cudaStreamDestroy(master);
    }
};

namespace {

using airg::fail;

// offsets inside a problem's dv buffer
struct Off {
    int m;
    size_t h1() const { return 0; }
    size_t h2() const { return size_t(m + 2); }
    size_t nrm() const { return size_t(2 * (m + 2)); }
    size_t bn() const { return nrm() + 1; }
    size_t rn() const { return nrm() + 2; }
    size_t y() const { return nrm() + 3; }
    size_t total() const { return y() + size_t(m) + 1; }
};

template <class F>
airg_status guarded(F&& f)
{
    try {
        f();
        airg::set_last_error("");
        return AIRG_OK;
    } catch (const airg::Error& e) {
        airg::set_last_error(e.msg.c_str());
        return e.st;
    } catch (const std::bad_alloc&) {
        airg::set_last_error("host allocation failed");
        return AIRG_ERR_OOM;
    } catch (const std::exception& e) {
        airg::set_last_error(e.what());
        return AIRG_ERR_STATE;
    }
}

void sync_all(airg_batch_s& B)
{
    for (cudaStream_t s : B.ps) CK(cudaStreamSynchronize(s));
    CK(cudaStreamSynchronize(B.master));
}

// graph of iteration j for all problems (captured on the master stream)
cudaGraphExec_t capture_iteration(airg_batch_s& B, int j)
{
    const int P = int(B.H.size());
    Off o{B.m};
    CK(cudaStreamBeginCapture(B.master, cudaStreamCaptureModeThreadLocal));
    try {
        CK(cudaEventRecord(B.fork, B.master));
        for (int p = 0; p < P; ++p) {
            airg::Hierarchy& H = *B.H[p];
            airg::SolveData& S = *H.solve;
            cudaStream_t st = B.ps[p];
            long long n = S.n0;
            double* dv = B.dv[p].p;
            CK(cudaStreamWaitEvent(st, B.fork, 0));
            double* vj = S.V.p + size_t(j) * n;
            double* zj = S.Zs.p + size_t(j) * n;
            if (j > 0) airg::mp_scale_dev(H, S.w.p, dv + o.nrm(), B.act[p].p, vj, st);
            airg::mp_vcycle(H, vj, zj, st);
            airg::mp_top_spmv(H, zj, S.w.p, st);
            airg::mp_multidot(H, j + 1, S.V.p, S.w.p, dv + o.h1(), 1, st);
            airg::mp_multiaxpy_norm(H, j + 1, S.V.p, dv + o.h1(), S.w.p, dv + o.nrm(), st);
            CK(cudaEventRecord(B.join[p], st));
            CK(cudaStreamWaitEvent(B.master, B.join[p], 0));
        }
    } catch (...) {
        cudaGraph_t g0;
        cudaStreamEndCapture(B.master, &g0);
        if (g0) cudaGraphDestroy(g0);
        throw;
    }
    cudaGraph_t graph;
    CK(cudaStreamEndCapture(B.master, &graph));
    cudaGraphExec_t exec;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    return exec;
}

// graph of one Richardson iteration for all problems: per problem
//     z = V-cycle(r) -> x += z (if active) -> r = b - A x -> <r, r>
cudaGraphExec_t capture_richardson(airg_batch_s& B)
{
    const int P = int(B.H.size());
    Off o{B.m};
    CK(cudaStreamBeginCapture(B.master, cudaStreamCaptureModeThreadLocal));
    try {
        CK(cudaEventRecord(B.fork, B.master));
        for (int p = 0; p < P; ++p) {
            airg::Hierarchy& H = *B.H[p];
            airg::SolveData& S = *H.solve;
            cudaStream_t st = B.ps[p];
            double* dv = B.dv[p].p;
            CK(cudaStreamWaitEvent(st, B.fork, 0));
            airg::mp_vcycle(H, S.r.p, S.Zs.p, st);
            airg::mp_add_dev(H, S.Zs.p, B.act[p].p, S.xp.p, st);
            airg::mp_residual(H, S.bp.p, S.xp.p, S.w.p, S.r.p, st);
            airg::mp_multidot(H, 0, S.V.p, S.r.p, dv + o.rn(), 1, st);
            CK(cudaEventRecord(B.join[p], st));
            CK(cudaStreamWaitEvent(B.master, B.join[p], 0));
        }
    } catch (...) {
        cudaGraph_t g0;
        cudaStreamEndCapture(B.master, &g0);
        if (g0) cudaGraphDestroy(g0);
        throw;
    }
    cudaGraph_t graph;
    CK(cudaStreamEndCapture(B.master, &graph));
    cudaGraphExec_t exec;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    return exec;
}

// Iteration j of all problems as one persistent work-list launch, captured
// (counter reset + kernel) in a graph of its own.
cudaGraphExec_t capture_worklist(airg_batch_s& B, int j)
{
    Off o{B.m};
    if (!B.wls[j]) {
        std::vector<airg::WlProblem> probs;
        for (size_t p = 0; p < B.H.size(); ++p)
            probs.push_back(airg::WlProblem{B.H[p].get(), B.dv[p].p + o.h1(), B.dv[p].p + o.nrm(), B.act[p].p});
        B.wls[j] = airg::build_worklist(probs, j, B.master);
    }
    CK(cudaStreamBeginCapture(B.master, cudaStreamCaptureModeThreadLocal));
    try {
        airg::launch_worklist(*B.wls[j], B.master);
    } catch (...) {
        cudaGraph_t g0;
        cudaStreamEndCapture(B.master, &g0);
        if (g0) cudaGraphDestroy(g0);
        throw;
    }
    cudaGraph_t graph;
    CK(cudaStreamEndCapture(B.master, &graph));
    cudaGraphExec_t exec;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    return exec;
}

long long iteration_bytes_of(airg_batch_s& B, int p, int j)
{
    if (B.it_bytes.size() <= size_t(j)) B.it_bytes.resize(size_t(j) + 1);
    std::vector<long long>& v = B.it_bytes[size_t(j)];
    if (v.empty()) {
        Off o{B.m};
        for (size_t q = 0; q < B.H.size(); ++q)
            v.push_back(airg::iteration_bytes(
                airg::WlProblem{B.H[q].get(), B.dv[q].p + o.h1(), B.dv[q].p + o.nrm(), B.act[q].p}, j));
    }
    return v[size_t(p)];
}

// Form of the lockstep FGMRES iteration: one graph with a branch per
// problem (default: measured faster on the 32-grid workload, 64.4 against
// 66.8 ms per solve), or with AIRG_MULTI=worklist the persistent work list
// where every hierarchy's layout allows it.
bool use_worklist(const airg_batch_s& B)
{
    const char* e = getenv("AIRG_MULTI");
    if (!e || std::strcmp(e, "worklist") != 0) return false;
    std::vector<airg::Hierarchy*> hs;
    for (const auto& H : B.H) hs.push_back(H.get());
    return airg::worklist_supported(hs);
}

void read_all(airg_batch_s& B, cudaStream_t st)
{
    Off o{B.m};
    size_t tot = o.total();
    for (size_t p = 0; p < B.H.size(); ++p)
        CK(cudaMemcpyAsync(B.hbuf.p + p * tot, B.dv[p].p, tot * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
}

struct PState {
    std::vector<double> Hm, cs, sn, g, y;
    double tol = 0, bn = 0, rn = 0;
    int active = 0, jdone = 0, its = 0;
};

void solve_multi(airg_batch_s& B, const double* const* b, double* const* x, bool on_device,
                 double rtol, double atol, int maxit, airg_solve_info* infos, cudaStream_t caller)
{
    auto t0 = std::chrono::steady_clock::now();
    const int P = int(B.H.size());
    const int m = B.m;
    Off o{m};
    const size_t tot = o.total();
    // order after the caller's stream
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, caller));
    for (cudaStream_t s : B.ps) CK(cudaStreamWaitEvent(s, ev, 0));
    CK(cudaStreamWaitEvent(B.master, ev, 0));
    CK(cudaEventDestroy(ev));
    std::vector<airg::DBuf<double>>& hb = B.stage_b;
    std::vector<airg::DBuf<double>>& hx = B.stage_x;
    std::vector<PState> st(P);
    // kernel launches per problem: the ones issued eagerly, plus every
    // graph launch's kernels; the captures themselves run nothing
    std::vector<long long> l0(P), cap(P, 0), run(P, 0);
    for (int p = 0; p < P; ++p) l0[p] = B.H[p]->solve->launches;
    auto counted = [&](std::vector<long long>& k, auto&& capture) {
        k.assign(size_t(P), 0);
        for (int p = 0; p < P; ++p) k[p] = -B.H[p]->solve->launches;
        cudaGraphExec_t g = capture();
        for (int p = 0; p < P; ++p) {
            k[p] += B.H[p]->solve->launches;
            cap[p] += k[p];
        }
        return g;
    };
    // inputs into the nested order, norms of b and of the first residual
    for (int p = 0; p < P; ++p) {
        airg::Hierarchy& H = *B.H[p];
        airg::SolveData& S = *H.solve;
        long long n = S.n0;
        const double* bd = b[p];
        const double* xd = x[p];
        if (!on_device) {
            if (hb[p].n < size_t(n)) hb[p].alloc(size_t(n));
            if (hx[p].n < size_t(n)) hx[p].alloc(size_t(n));
            airg::h2d(hb[p].p, b[p], size_t(n), B.ps[p]);
            airg::h2d(hx[p].p, x[p], size_t(n), B.ps[p]);
            bd = hb[p].p;
            xd = hx[p].p;
        }
        airg::mp_permute(H, bd, S.bp.p, true, B.ps[p]);
        airg::mp_permute(H, xd, S.xp.p, true, B.ps[p]);
        airg::mp_multidot(H, 0, S.V.p, S.bp.p, B.dv[p].p + o.bn(), 1, B.ps[p]);
        airg::mp_residual(H, S.bp.p, S.xp.p, S.w.p, S.r.p, B.ps[p]);
        airg::mp_multidot(H, 0, S.V.p, S.r.p, B.dv[p].p + o.rn(), 1, B.ps[p]);
        st[p].Hm.assign(size_t(m + 1) * m, 0.0);
        st[p].cs.assign(m, 0.0);
        st[p].sn.assign(m, 0.0);
        st[p].g.assign(size_t(m) + 1, 0.0);
        st[p].y.assign(size_t(m), 0.0);
    }
    sync_all(B);
    read_all(B, B.master);
    for (int p = 0; p < P; ++p) {
        st[p].bn = std::sqrt(std::max(B.hbuf.p[p * tot + o.bn()], 0.0));
        st[p].rn = std::sqrt(std::max(B.hbuf.p[p * tot + o.rn()], 0.0));
        st[p].tol = std::max(rtol * st[p].bn, atol);
    }
    int its = 0;
    const bool rich = B.H[0]->opt.outer == AIRG_OUTER_RICHARDSON;
    const bool wl = !rich && use_worklist(B);
    while (rich && its < maxit) {
        // lockstep Richardson; a converged problem keeps its x
        int nact = 0;
        for (int p = 0; p < P; ++p) {
            st[p].active = st[p].rn > st[p].tol;
            nact += st[p].active;
            airg::h2d(B.act[p].p, &st[p].active, 1, B.ps[p]);
        }
        sync_all(B);
        if (!nact) break;
        if (!B.rich) B.rich = counted(B.rk, [&] { return capture_richardson(B); });
        CK(cudaGraphLaunch(B.rich, B.master));
        for (int p = 0; p < P; ++p) run[p] += B.rk[p];
        read_all(B, B.master);
        ++its;
        for (int p = 0; p < P; ++p) {
            if (st[p].active) st[p].its += 1;
            st[p].rn = std::sqrt(std::max(B.hbuf.p[p * tot + o.rn()], 0.0));
        }
    }
    while (!rich && its < maxit) {
        int nact = 0;
        for (int p = 0; p < P; ++p) {
            PState& s = st[p];
            s.active = s.rn > s.tol;
            s.jdone = 0;
            nact += s.active;
            std::fill(s.g.begin(), s.g.end(), 0.0);
            s.g[0] = s.rn;
            airg::h2d(B.act[p].p, &s.active, 1, B.ps[p]);
            airg::SolveData& S = *B.H[p]->solve;
            // v_0 = r / ||r|| (the squared norm is on the device already)
            airg::mp_scale_dev(*B.H[p], S.r.p, B.dv[p].p + o.rn(), B.act[p].p, S.V.p, B.ps[p]);
        }
        sync_all(B);
        if (!nact) break;
        for (int j = 0; j < m; ++j) {
            if (wl && !B.wgraphs[j]) B.wgraphs[j] = capture_worklist(B, j);
            if (!wl && !B.graphs[j]) B.graphs[j] = counted(B.gk[j], [&] { return capture_iteration(B, j); });
            if (B.prof) CK(cudaEventRecord(B.pev[0], B.master));
            if (wl) {
                CK(cudaGraphLaunch(B.wgraphs[j], B.master));
                run[0] += 1;   // one kernel for all problems
            } else {
                CK(cudaGraphLaunch(B.graphs[j], B.master));
                for (int p = 0; p < P; ++p) run[p] += B.gk[j][p];
            }
            if (B.prof) CK(cudaEventRecord(B.pev[1], B.master));
            read_all(B, B.master);
            if (B.prof) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, B.pev[0], B.pev[1]));
                B.prof_ms += ms;
                B.prof_launches += 1;
                for (int p = 0; p < P; ++p)
                    if (st[p].active) B.prof_bytes += iteration_bytes_of(B, p, j);
            }
            ++its;
            // second Gram-Schmidt pass where the first cancelled too much
            bool again = false;
            for (int p = 0; p < P; ++p) {
                const double* hp = B.hbuf.p + p * tot;
                if (!st[p].active || !(hp[o.nrm()] < airg::reorth_ratio() * hp[o.h1() + j + 1])) continue;
                airg::Hierarchy& H = *B.H[p];
                airg::SolveData& S = *H.solve;
                airg::mp_multidot(H, j + 1, S.V.p, S.w.p, B.dv[p].p + o.h2(), 0, B.ps[p]);
                airg::mp_multiaxpy_norm(H, j + 1, S.V.p, B.dv[p].p + o.h2(), S.w.p, B.dv[p].p + o.nrm(),
                                        B.ps[p]);
                again = true;
            }
            std::vector<double> first;
            if (again) {
                first.assign(B.hbuf.p, B.hbuf.p + size_t(P) * tot);
                sync_all(B);
                read_all(B, B.master);
            }
            int still = 0;
            for (int p = 0; p < P; ++p) {
                PState& s = st[p];
                if (!s.active) continue;
                const double* hp = B.hbuf.p + p * tot;
                const double* h1 = again ? first.data() + p * tot : hp;
                auto h = [&](int i, int c) -> double& { return s.Hm[size_t(i) * m + c]; };
                bool two = again && (h1[o.nrm()] < airg::reorth_ratio() * h1[o.h1() + j + 1]);
                for (int i = 0; i <= j; ++i) h(i, j) = h1[o.h1() + i] + (two ? hp[o.h2() + i] : 0.0);
                double hn = std::sqrt(std::max(hp[o.nrm()], 0.0));
                h(j + 1, j) = hn;
                for (int i = 0; i < j; ++i) {
                    double a = h(i, j), c = h(i + 1, j);
                    h(i, j) = s.cs[i] * a + s.sn[i] * c;
                    h(i + 1, j) = -s.sn[i] * a + s.cs[i] * c;
                }
                double a = h(j, j), c = h(j + 1, j);
                double den = std::hypot(a, c);
                s.cs[j] = den > 0 ? a / den : 1.0;
                s.sn[j] = den > 0 ? c / den : 0.0;
                h(j, j) = den;
                h(j + 1, j) = 0.0;
                s.g[j + 1] = -s.sn[j] * s.g[j];
                s.g[j] = s.cs[j] * s.g[j];
                s.jdone = j + 1;
                s.its += 1;
                if (std::fabs(s.g[j + 1]) <= s.tol || den == 0.0 || hn == 0.0) s.active = 0;
                else ++still;
            }
            if (!still || its >= maxit || j + 1 == m) break;
            for (int p = 0; p < P; ++p) airg::h2d(B.act[p].p, &st[p].active, 1, B.ps[p]);
            sync_all(B);
        }
        // x += Z y per problem, then the true residual
        for (int p = 0; p < P; ++p) {
            PState& s = st[p];
            airg::Hierarchy& H = *B.H[p];
            airg::SolveData& S = *H.solve;
            int jd = s.jdone;
            auto h = [&](int i, int c) -> double { return s.Hm[size_t(i) * m + c]; };
            for (int j = jd - 1; j >= 0; --j) {
                double v = s.g[j];
                for (int i = j + 1; i < jd; ++i) v -= h(j, i) * s.y[i];
                s.y[j] = v / h(j, j);
            }
            if (jd) {
                airg::h2d(B.dv[p].p + o.y(), s.y.data(), size_t(jd), B.ps[p]);
                airg::mp_update(H, jd, S.Zs.p, B.dv[p].p + o.y(), S.xp.p, B.ps[p]);
            }
            airg::mp_residual(H, S.bp.p, S.xp.p, S.w.p, S.r.p, B.ps[p]);
            airg::mp_multidot(H, 0, S.V.p, S.r.p, B.dv[p].p + o.rn(), 1, B.ps[p]);
        }
        sync_all(B);
        read_all(B, B.master);
        for (int p = 0; p < P; ++p) st[p].rn = std::sqrt(std::max(B.hbuf.p[p * tot + o.rn()], 0.0));
    }
    bool all = true;
    for (int p = 0; p < P; ++p) {
        airg::Hierarchy& H = *B.H[p];
        airg::SolveData& S = *H.solve;
        long long n = S.n0;
        double* xd = on_device ? x[p] : hx[p].p;
        airg::mp_permute(H, S.xp.p, xd, false, B.ps[p]);
        if (!on_device) CK(cudaMemcpyAsync(x[p], hx[p].p, sizeof(double) * n, cudaMemcpyDeviceToHost, B.ps[p]));
        bool conv = st[p].rn <= st[p].tol;
        all = all && conv;
        if (infos) {
            infos[p].iterations = st[p].its;
            infos[p].rel_residual = st[p].bn > 0 ? st[p].rn / st[p].bn : 0.0;
            infos[p].converged = conv;
            infos[p].kernel_launches = B.H[p]->solve->launches - l0[p] - cap[p] + run[p];
        }
    }
    sync_all(B);
    bool gave_up = false;
    for (auto& w : B.wls)
        if (w && airg::worklist_timed_out(*w, B.master)) gave_up = true;
    if (gave_up) fail(AIRG_ERR_TIMEOUT, "a wait of the work-list kernel gave up");
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (infos)
        for (int p = 0; p < P; ++p) infos[p].solve_ms = ms;
    if (!all) fail(AIRG_ERR_NOT_CONVERGED, "a problem of the batch did not reach the tolerance within maxit");
}

}  // namespace

extern "C" {

airg_status airg_setup_batch(int nprob, const airg_csr* As, const airg_options* opt, void* stream,
                             airg_batch** out)
{
    return guarded([&] {
        if (!out || nprob < 1 || !As) fail(AIRG_ERR_ARG, "bad batch setup arguments");
        *out = nullptr;
        airg_options o;
        if (opt) o = *opt;
        else airg_options_default(&o);
        airg::check_options_checked(o);
        cudaStream_t st = (cudaStream_t)stream;
        auto B = std::make_unique<airg_batch_s>();
        for (int p = 0; p < nprob; ++p) {
            airg::DevCSR D = airg::upload_csr_checked(&As[p], st);
            B->H.push_back(airg::build_hierarchy(std::move(D), o, st));
        }
        B->m = B->H[0]->solve->restart;
        Off of{B->m};
        for (int p = 0; p < nprob; ++p) {
            cudaStream_t s;
            CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            B->ps.push_back(s);
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            B->join.push_back(e);
            airg::DBuf<double> d(of.total());
            CK(cudaMemset(d.p, 0, d.bytes()));
            B->dv.push_back(std::move(d));
            airg::DBuf<int> a(1);
            CK(cudaMemset(a.p, 0, sizeof(int)));
            B->act.push_back(std::move(a));
        }
        CK(cudaStreamCreateWithFlags(&B->master, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
        B->hbuf.alloc(size_t(nprob) * of.total());
        B->graphs.assign(size_t(B->m), nullptr);
        B->gk.assign(size_t(B->m), {});
        B->wls.assign(size_t(B->m), nullptr);
        B->wgraphs.assign(size_t(B->m), nullptr);
        B->stage_b.resize(size_t(nprob));
        B->stage_x.resize(size_t(nprob));
        *out = B.release();
    });
}

airg_status airg_solve_batch(airg_batch* b, const double* const* bvec, double* const* xvec, int on_device,
                             double rtol, double atol, int maxit, airg_solve_info* infos, void* stream)
{
    return guarded([&] {
        if (!b || !bvec || !xvec || maxit < 0 || !(rtol >= 0.0) || !(atol >= 0.0))
            fail(AIRG_ERR_ARG, "bad batch solve arguments");
        for (size_t p = 0; p < b->H.size(); ++p)
            if (!bvec[p] || !xvec[p]) fail(AIRG_ERR_ARG, "null vector in the batch");
        solve_multi(*b, bvec, xvec, on_device != 0, rtol, atol, maxit, infos, (cudaStream_t)stream);
    });
}

airg_status airg_batch_profile(airg_batch* b, int enable)
{
    return guarded([&] {
        if (!b) fail(AIRG_ERR_ARG, "null batch");
        for (cudaEvent_t& e : b->pev)
            if (!e) CK(cudaEventCreate(&e));
        b->prof = enable != 0;
        b->prof_ms = 0.0;
        b->prof_launches = b->prof_bytes = 0;
    });
}

airg_status airg_batch_profile_read(const airg_batch* b, double* ms, int64_t* launches, int64_t* bytes)
{
    return guarded([&] {
        if (!b || !ms || !launches || !bytes) fail(AIRG_ERR_ARG, "bad batch profile arguments");
        *ms = b->prof_ms;
        *launches = b->prof_launches;
        *bytes = b->prof_bytes;
    });
}

airg_status airg_batch_setup_info(const airg_batch* b, int i, airg_hierarchy_info* info)
{
    return guarded([&] {
        if (!b || !info || i < 0 || size_t(i) >= b->H.size()) fail(AIRG_ERR_ARG, "bad batch index or info");
        airg::fill_setup_info(*b->H[size_t(i)], info);
    });
}

void airg_batch_free(airg_batch* b) { delete b; }

}  // extern "C"

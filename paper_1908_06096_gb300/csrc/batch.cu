// Batched execution of many plans: one launch per stage for all requests,
// optionally replayed from a captured CUDA graph (include/st.h, st_batch_*).
#include "st_internal.cuh"

#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <string>

using namespace st;

struct st_batch {
    // per precision: the jobs of each stage (chunks of at most MAX_JOBS)
    struct Stage {
        std::vector<PackJob> pack, unpack;
        std::vector<TcJob> tc_inv, tc_dir;
        std::vector<SimtJob> simt_inv, simt_dir;
        std::vector<long long> simt_inv_blocks, simt_dir_blocks;
        std::vector<FftJob> fft_inv, fft_dir;
        std::vector<FftJob> fft_inv_w, fft_dir_w;  // the same rows within a half CTA's shared memory
        std::vector<std::pair<st_plan *, int>> tf32_dir;  // 3xTF32 direct items: operand transposes
        size_t smem_inv = 0, smem_dir = 0;
        int var_inv = 0, var_dir = 0;  // launch variant of the largest job
        long long big_inv = -1, big_dir = -1;
    };
    std::map<int, Stage> by_prec;
    int sm_count = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    PersState *pers = nullptr;  // the persistent kernel's tables, when the batch qualifies
    std::string pers_why;       // why it does not
    int *err = nullptr;
};

namespace {

long long fft_ctas(const std::vector<FftJob> &jobs)
{
    long long n = 0;
    for (const FftJob &J : jobs) n += (long long)J.J * J.nfg;
    return n;
}

template <class J, class F>
st_status chunked(const std::vector<J> &v, F f)
{
    for (size_t i = 0; i < v.size(); i += MAX_JOBS) {
        const int n = (int)std::min<size_t>(MAX_JOBS, v.size() - i);
        st_status r = f(v.data() + i, n, i);
        if (r) return r;
    }
    return ST_OK;
}

st_status batch_launch(st_batch *b, cudaStream_t s)
{
    st_status r;
    for (auto &kv : b->by_prec) {
        const int prec = kv.first;
        auto &S = kv.second;
        if ((r = chunked(S.pack, [&](const PackJob *j, int n, size_t) { return launch_pack_jobs(0, prec, j, n, s); })))
            return r;
        if ((r = chunked(S.tc_inv, [&](const TcJob *j, int n, size_t) { return launch_tc_jobs(prec, j, n, b->sm_count, s); })))
            return r;
        if ((r = chunked(S.simt_inv, [&](const SimtJob *j, int n, size_t i) {
                 return launch_simt_jobs(prec, j, S.simt_inv_blocks.data() + i, n, s);
             })))
            return r;
        if ((r = chunked(S.fft_inv, [&](const FftJob *j, int n, size_t) {
                 return launch_fft_jobs(0, prec, j, n, S.smem_inv, s, S.var_inv);
             })))
            return r;
    }
    for (auto &kv : b->by_prec) {
        const int prec = kv.first;
        auto &S = kv.second;
        if ((r = chunked(S.fft_dir, [&](const FftJob *j, int n, size_t) {
                 return launch_fft_jobs(1, prec, j, n, S.smem_dir, s, S.var_dir);
             })))
            return r;
        for (auto &pn : S.tf32_dir)
            if ((r = launch_fb_tf32split(pn.first, pn.second, s))) return r;
        if ((r = chunked(S.tc_dir, [&](const TcJob *j, int n, size_t) { return launch_tc_jobs(prec, j, n, b->sm_count, s); })))
            return r;
        if ((r = chunked(S.simt_dir, [&](const SimtJob *j, int n, size_t i) {
                 return launch_simt_jobs(prec, j, S.simt_dir_blocks.data() + i, n, s);
             })))
            return r;
        if ((r = chunked(S.unpack, [&](const PackJob *j, int n, size_t) { return launch_pack_jobs(1, prec, j, n, s); })))
            return r;
    }
    return ST_OK;
}

// A job the persistent kernel refuses (its rows did not fit a wide CTA).
FftJob no_wide_job()
{
    FftJob J;
    memset(&J, 0, sizeof(J));
    J.kind = -1;
    return J;
}

// Per-CTA shared-memory budget of the row-FFT jobs of the persistent kernel:
// each half of its CTA holds one job's CTA, within FF_HALF_BYTES.
int wide_kb(const st_plan *p, int dir) { return std::min(FF_HALF_BYTES / 1024 - 4, p->fft_kb[dir]); }

// Tables of the persistent kernel, when the batch is one tensor-core
// precision whose rows all have compile-time FFT plans; else the reason.
void persistent_setup(st_batch *b)
{
    if (b->by_prec.size() != 1) {
        b->pers_why = "it mixes precisions";
        return;
    }
    auto &kv = *b->by_prec.begin();
    auto &S = kv.second;
    PersInput in;
    in.prec = kv.first;
    in.sm_count = b->sm_count;
    in.err = b->err;
    in.pack = S.pack;
    in.unpack = S.unpack;
    in.tc_inv = S.tc_inv;
    in.tc_dir = S.tc_dir;
    in.fft_inv = S.fft_inv_w;
    in.fft_dir = S.fft_dir_w;
    if (pers_prepare(in, &b->pers) != ST_OK) {
        b->pers = nullptr;
        b->pers_why = st_last_error();
    }
}

}  // namespace

extern "C" {

st_status st_batch_create(st_batch_t *out, const st_batch_item *items, int n)
{
    if (!out) return ST_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !items) return ST_ERR_ARG;
    std::set<st_plan_t> seen;
    for (int i = 0; i < n; ++i) {
        const st_batch_item &it = items[i];
        if (!it.plan || it.direction < 0 || it.direction > 2 || it.nfields < 1 || it.nfields > it.plan->max_fields ||
            !it.grid || (it.direction != 1 && !it.spec_in) || (it.direction != 0 && !it.spec_out)) {
            set_last_error("invalid batch item " + std::to_string(i));
            return ST_ERR_ARG;
        }
        if (!seen.insert(it.plan).second) {
            set_last_error("a plan appears in more than one batch item");
            return ST_ERR_BUSY;
        }
    }
    st_batch *b = new st_batch();
    b->sm_count = items[0].plan->sm_count;
    for (int i = 0; i < n; ++i) {
        const st_batch_item &it = items[i];
        st_plan *p = it.plan;
        auto &S = b->by_prec[p->prec];
        st_status r = ST_OK;
        if (it.direction != 1) {
            PackJob pj;
            pack_job(p, 0, it.nfields, it.spec_in, p->sop, &pj);
            S.pack.push_back(pj);
            if (prec_is_tc(p->prec)) {
                TcJob tj;
                if ((r = tc_job(p, 0, it.nfields, p->sop, p->fb, &tj))) { delete b; return r; }
                S.tc_inv.push_back(tj);
            } else {
                SimtJob sj;
                long long blocks = 0;
                simt_job(p, 0, it.nfields, p->sop, p->fb, &sj, &blocks);
                S.simt_inv.push_back(sj);
                S.simt_inv_blocks.push_back(blocks);
            }
            std::vector<FftJob> fj;
            size_t smem = 0;
            if ((r = fft_jobs(p, 0, it.nfields, p->fb, it.grid, fj, &smem))) { delete b; return r; }
            S.fft_inv.insert(S.fft_inv.end(), fj.begin(), fj.end());
            if (p->prec != P_FP64) {
                std::vector<FftJob> fw;
                size_t sw = 0;
                if (fft_jobs(p, 0, it.nfields, p->fb, it.grid, fw, &sw, wide_kb(p, 0)) == ST_OK)
                    S.fft_inv_w.insert(S.fft_inv_w.end(), fw.begin(), fw.end());
                else
                    S.fft_inv_w.push_back(no_wide_job());
            }
            S.smem_inv = std::max(S.smem_inv, smem);
            const long long ctas = fft_ctas(fj);
            if (ctas > S.big_inv) { S.big_inv = ctas; S.var_inv = p->fft_var[0]; }
        }
        if (it.direction != 0) {
            std::vector<FftJob> fj;
            size_t smem = 0;
            if ((r = fft_dir_jobs(p, it.nfields, it.grid, fj, &smem))) { delete b; return r; }
            S.fft_dir.insert(S.fft_dir.end(), fj.begin(), fj.end());
            if (p->prec == P_TF32X3) S.tf32_dir.emplace_back(p, it.nfields);
            if (p->prec != P_FP64) {
                std::vector<FftJob> fw;
                size_t sw = 0;
                if (fft_dir_jobs(p, it.nfields, it.grid, fw, &sw, wide_kb(p, 1)) == ST_OK)
                    S.fft_dir_w.insert(S.fft_dir_w.end(), fw.begin(), fw.end());
                else
                    S.fft_dir_w.push_back(no_wide_job());
            }
            S.smem_dir = std::max(S.smem_dir, smem);
            const long long ctas = fft_ctas(fj);
            if (ctas > S.big_dir) { S.big_dir = ctas; S.var_dir = p->fft_var[1]; }
            if (prec_is_tc(p->prec)) {
                TcJob tj;
                if ((r = tc_job(p, 1, it.nfields, p->fbop, p->sout, &tj))) { delete b; return r; }
                S.tc_dir.push_back(tj);
            } else {
                SimtJob sj;
                long long blocks = 0;
                simt_job(p, 1, it.nfields, p->fbop, p->sout, &sj, &blocks);
                S.simt_dir.push_back(sj);
                S.simt_dir_blocks.push_back(blocks);
            }
            PackJob uj;
            pack_job(p, 1, it.nfields, p->sout, it.spec_out, &uj);
            S.unpack.push_back(uj);
        }
    }
    b->err = items[0].plan->err;
    persistent_setup(b);
    *out = b;
    return ST_OK;
}

st_status st_batch_run(st_batch_t b, void *stream, int use_graph)
{
    if (!b) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (use_graph == 2) {
        if (!b->pers) {
            set_last_error("this batch does not run as one persistent launch: " + b->pers_why);
            return ST_ERR_UNSUPPORTED;
        }
        return pers_launch(b->pers, s);
    }
    if (!use_graph) return batch_launch(b, s);
    if (!b->exec) {
        // record on a private stream (the legacy default stream cannot be
        // captured); recording runs nothing, the graph then runs on `s`
        if (!b->cap) ST_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        ST_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        st_status r = batch_launch(b, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (r != ST_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        b->graph = g;
    }
    ST_CUDA(cudaGraphLaunch(b->exec, s));
    return ST_OK;
}

st_status st_batch_destroy(st_batch_t b)
{
    if (!b) return ST_OK;
    pers_free(b->pers);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return ST_OK;
}

}  // extern "C"

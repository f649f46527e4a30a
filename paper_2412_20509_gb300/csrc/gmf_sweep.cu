// Batched rank sweep: several GMF fits of different latent rank d on the same
// count matrix (the model-selection use of Sec. 4.2, where d must be chosen
// from a grid of fits). Model 0 owns the permuted counts; the others read them.
// The models, heaviest first, are split into groups of `group`; per sweep, one
// tile launch covers every model of a group (grid z = model slot x block, the
// heaviest models in the lowest slots so their CTAs start first) and one update
// launch covers their strips; a whole epoch of these launches is captured once
// into a CUDA graph. gmf_sweep_autotune times the groupings on trial sweeps
// (the models' state is saved before and restored after) and keeps the
// fastest; every grouping gives the same results bit for bit.
#include <algorithm>
#include <string>
#include <vector>

#include "gmf_internal.cuh"

// gmf_step_tc.cu / gmf_step_simt.cu
size_t gmf_tc_layout_size();
const void* gmf_tc_layout(const gmf_model* h);
uint32_t gmf_tc_smem(const gmf_model* h);
uint32_t gmf_tc_tmem_cols(const gmf_model* h);
void gmf_tc_grid(const gmf_model* h, int* TI, int* TJ);
cudaError_t gmf_tc_multi_attr(const gmf_model* h0, uint32_t smem);
cudaError_t gmf_tc_launch_multi(const gmf_model* h0, const StepArgs* d_args, const void* d_lays, const int* d_order,
                                int nmodels, uint32_t smem, int w, cudaStream_t st);
cudaError_t gmf_tc_launch_multi_persist(const gmf_model* h0, const StepArgs* d_args, const void* d_lays,
                                        const int* d_order, int nmodels, uint32_t smem, uint32_t tmem_cols, int w,
                                        unsigned* gctr, unsigned* err, cudaStream_t st);
size_t gmf_sweep_simt_smem(const gmf_model* h);
cudaError_t gmf_simt_multi_attr(size_t smem);
cudaError_t gmf_simt_launch_multi(const gmf_model* h0, const StepArgs* d_args, const int* d_order, int nmodels,
                                  size_t smem, int w, cudaStream_t st);

extern "C" int gmf_sgd_sweeps(gmf_model* h, const int32_t* sigma, int32_t w_begin, int32_t w_end, void* stream);

struct gmf_sweep {
    std::vector<gmf_model*> models;
    std::vector<int> order;        // model of each slot, heaviest first
    std::vector<size_t> slot_smem; // tile launch shared memory of each slot's model
    StepArgs* d_args = nullptr;    // per slot
    void* d_lays = nullptr;        // per slot (tensor-core layouts)
    int* d_order = nullptr;        // identity: slot -> its own argument entry
    int group = 0;                 // models per launch (0: all; GMF_SWEEP_SEQUENTIAL: model after model)
    size_t smem = 0;
    uint32_t tmem_cols = 0;        // TMEM columns of the widest model's tile (persistent launch)
    size_t upd_smem = 0;   // update launch: the largest model's staging
    int upd_units = 0;     // update launch: CTAs per model
    int upd_threads = 0;   // tensor-core update launch: threads per CTA (the widest model's)
    int mixed = 0;
    unsigned* gctr = nullptr;      // grid-barrier counter of the persistent launch
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap = nullptr;
};

static void sweep_release(gmf_sweep* s) {
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->d_args) cudaFree(s->d_args);
    if (s->d_lays) cudaFree(s->d_lays);
    if (s->d_order) cudaFree(s->d_order);
    if (s->gctr) cudaFree(s->gctr);
    for (size_t i = s->models.size(); i-- > 0;) gmf_free(s->models[i]);  // the owner of the counts last
    delete s;
}

extern "C" void gmf_sweep_free(gmf_sweep* s) { sweep_release(s); }

static int sweep_fail(gmf_sweep* s, int code, const std::string& msg) {
    sweep_release(s);
    return gmf_fail(code, msg.c_str());
}

extern "C" int gmf_sweep_init(gmf_sweep** out, const gmf_config* cfg, const int32_t* d_list, int32_t n_models,
                              const void* Y, int32_t y_dtype, int32_t y_on_device, const float* W, const double* X,
                              const double* Z, const double* offset, const int32_t* row_perm, const int32_t* col_perm,
                              const double* const* B0, const double* const* G0, const double* const* U0,
                              const double* const* V0, const double* alpha0, void* stream) {
    if (!out || !cfg || !d_list || !B0 || !G0 || !U0 || !V0 || !alpha0)
        return gmf_fail(GMF_ERR_ARG, "gmf_sweep_init: NULL argument");
    *out = nullptr;
    if (cfg->family > GMF_NEGBIN) return gmf_fail(GMF_ERR_STATE, "gmf_sweep_init: Poisson and negative binomial fits only");
    if (n_models < 1 || n_models > 64) return gmf_fail(GMF_ERR_ARG, "gmf_sweep_init: 1 <= n_models <= 64");
    gmf_sweep* s = new gmf_sweep();
    s->mixed = cfg->precision == GMF_PREC_MIXED;
    for (int i = 0; i < n_models; i++) {
        gmf_config c = *cfg;
        c.d = d_list[i];
        gmf_model* h = nullptr;
        const int rc = i == 0 ? gmf_init(&h, &c, Y, y_dtype, y_on_device, W, X, Z, offset, row_perm, col_perm, B0[i],
                                         G0[i], U0[i], V0[i], alpha0[i], stream)
                              : gmf_init_shared(&h, &c, s->models[0], X, Z, offset, B0[i], G0[i], U0[i], V0[i],
                                                alpha0[i], stream);
        if (rc != GMF_OK) {
            const std::string keep = gmf_last_error();
            return sweep_fail(s, rc, "gmf_sweep_init: model " + std::to_string(i) + ": " + keep);
        }
        s->models.push_back(h);
    }
    s->models[0]->y_fixed = 1;  // the other models read its count buffer
    // heaviest models first (per-entry work grows with K = 1+p+q+d)
    std::vector<int> order(n_models);
    for (int i = 0; i < n_models; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s->models[a]->K > s->models[b]->K; });
    s->order = order;
    std::vector<StepArgs> args(n_models);
    std::vector<char> lays;
    for (int i = 0; i < n_models; i++) {  // in slot order
        gmf_model* h = s->models[order[i]];
        args[i] = gmf_make_args(h);
        if (s->mixed) {
            gmf_tc_grid(h, &args[i].TI, &args[i].TJ);
            const char* l = (const char*)gmf_tc_layout(h);
            lays.insert(lays.end(), l, l + gmf_tc_layout_size());
            s->slot_smem.push_back(gmf_tc_smem(h));
            s->tmem_cols = std::max(s->tmem_cols, gmf_tc_tmem_cols(h));
        } else {
            s->slot_smem.push_back(gmf_sweep_simt_smem(h));
        }
        s->smem = std::max(s->smem, s->slot_smem.back());
        s->upd_smem = std::max(s->upd_smem, gmf_update_smem(args[i]));
    }
    s->upd_units = s->mixed ? gmf_update_tc_units(args[0], 128) : gmf_update_units(args[0], GMF_TILE);
    for (int i = 0; i < n_models; i++) s->upd_threads = std::max(s->upd_threads, gmf_update_tc_threads(args[i]));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMalloc(&s->d_args, sizeof(StepArgs) * n_models) != cudaSuccess ||
        cudaMalloc(&s->d_order, sizeof(int) * n_models) != cudaSuccess ||
        (s->mixed && cudaMalloc(&s->d_lays, lays.size()) != cudaSuccess) ||
        (s->mixed && cudaMalloc(&s->gctr, sizeof(unsigned)) != cudaSuccess))
        return sweep_fail(s, GMF_ERR_OOM, "gmf_sweep_init: device allocation failed");
    if (s->gctr) cudaMemsetAsync(s->gctr, 0, sizeof(unsigned), st);
    cudaMemcpyAsync(s->d_args, args.data(), sizeof(StepArgs) * n_models, cudaMemcpyHostToDevice, st);
    std::vector<int> ident(n_models);
    for (int i = 0; i < n_models; i++) ident[i] = i;
    cudaMemcpyAsync(s->d_order, ident.data(), sizeof(int) * n_models, cudaMemcpyHostToDevice, st);
    if (s->mixed) cudaMemcpyAsync(s->d_lays, lays.data(), lays.size(), cudaMemcpyHostToDevice, st);
    const cudaError_t e =
        s->mixed ? gmf_tc_multi_attr(s->models[0], (uint32_t)s->smem) : gmf_simt_multi_attr(s->smem);
    if (e != cudaSuccess)
        return sweep_fail(s, GMF_ERR_ARG, std::string("gmf_sweep_init: the largest model's tile does not fit: ") +
                                               cudaGetErrorString(e));
    if (cudaStreamSynchronize(st) != cudaSuccess) return sweep_fail(s, GMF_ERR_CUDA, "gmf_sweep_init: copy failed");
    *out = s;
    return GMF_OK;
}

// One sweep of every model: per group of slots [g0, g0 + gn), a tile launch and an update launch, or one
// persistent launch for all models.
static cudaError_t launch(gmf_sweep* s, int w, cudaStream_t st, int group) {
    const int nm = (int)s->models.size();
    if (group == GMF_SWEEP_PERSISTENT)
        return gmf_tc_launch_multi_persist(s->models[0], s->d_args, s->d_lays, s->d_order, nm, (uint32_t)s->smem,
                                           s->tmem_cols, w, s->gctr, s->models[0]->err, st);
    const int gsz = group > 0 ? std::min(group, nm) : nm;
    const size_t lay_bytes = s->mixed ? gmf_tc_layout_size() : 0;
    for (int g0 = 0; g0 < nm; g0 += gsz) {
        const int gn = std::min(gsz, nm - g0);
        const StepArgs* args = s->d_args + g0;
        // the group's own largest tile: small models launched alone keep their occupancy
        size_t smem = 0;
        for (int i = g0; i < g0 + gn; i++) smem = std::max(smem, s->slot_smem[i]);
        const cudaError_t e =
            s->mixed ? gmf_tc_launch_multi(s->models[0], args, (const char*)s->d_lays + g0 * lay_bytes, s->d_order, gn,
                                           (uint32_t)smem, w, st)
                     : gmf_simt_launch_multi(s->models[0], args, s->d_order, gn, smem, w, st);
        if (e != cudaSuccess) return e;
        const cudaError_t e2 =
            (s->mixed ? gmf_launch_update_tc_multi(args, gn, s->upd_units, s->upd_threads, w, 128, st)
                     : gmf_launch_update_multi(args, gn, s->upd_units, s->upd_smem, w, GMF_TILE, st));
        if (e2 != cudaSuccess) return e2;
    }
    return cudaSuccess;
}

extern "C" int gmf_sweep_epoch(gmf_sweep* s, const int32_t* sigma, void* stream) {
    if (!s || !sigma) return gmf_fail(GMF_ERR_ARG, "gmf_sweep_epoch: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    gmf_model* h0 = s->models[0];
    std::vector<char> seen(h0->nsw, 0);
    for (int w = 0; w < h0->nsw; w++) {
        if (sigma[w] < 0 || sigma[w] >= h0->nsw || seen[sigma[w]])
            return gmf_fail(GMF_ERR_ARG, "gmf_sweep_epoch: sigma is not a permutation");
        seen[sigma[w]] = 1;
    }
    if (s->group == GMF_SWEEP_SEQUENTIAL) {  // each model's own epoch (its single-model launches and graph)
        for (size_t i = 0; i < s->models.size(); i++) {
            const int rc = gmf_sgd_sweeps(s->models[s->order[i]], sigma, 0, h0->nsw, stream);
            if (rc) return rc;
        }
        return GMF_OK;
    }
    for (gmf_model* h : s->models) {
        const int rc = gmf_stage_schedule(h, sigma, 0, h->nsw, st);
        if (rc) return rc;
    }
    if (!s->graph) {
        if (!s->cap && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess)
            return gmf_fail(GMF_ERR_CUDA, "gmf_sweep_epoch: stream creation failed");
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return gmf_fail(GMF_ERR_CUDA, "gmf_sweep_epoch: capture failed");
        cudaError_t e = cudaSuccess;
        if (s->group == GMF_SWEEP_PERSISTENT) e = cudaMemsetAsync(s->gctr, 0, sizeof(unsigned), s->cap);
        for (int w = 0; w < h0->nsw && e == cudaSuccess; w++) e = launch(s, w, s->cap, s->group);
        const cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
        if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            s->graph = nullptr;
            return gmf_fail(GMF_ERR_CUDA, "gmf_sweep_epoch: graph capture of the sweep launches failed");
        }
    }
    if (cudaGraphLaunch(s->graph, st) != cudaSuccess) return gmf_fail(GMF_ERR_CUDA, "gmf_sweep_epoch: launch failed");
    for (gmf_model* h : s->models) h->t += (int64_t)h->nsw * h->per;
    return GMF_OK;
}

extern "C" int gmf_sweep_set_group(gmf_sweep* s, int32_t group) {
    if (!s || ((group < GMF_SWEEP_SEQUENTIAL || group > (int32_t)s->models.size()) &&
               !(group == GMF_SWEEP_PERSISTENT && s->mixed)))
        return gmf_fail(GMF_ERR_ARG, "gmf_sweep_set_group: group outside [-1, n_models] (or a persistent launch on "
                                     "the FP32 path)");
    if (group != s->group && s->graph) {
        cudaGraphExecDestroy(s->graph);  // recaptured by the next epoch
        s->graph = nullptr;
    }
    s->group = group;
    return GMF_OK;
}

extern "C" int32_t gmf_sweep_group(const gmf_sweep* s) {
    if (!s) return -2;
    return s->group != 0 ? s->group : (int32_t)s->models.size();
}

// The device state a sweep changes, per model: parameters, smoothed derivatives,
// visit counts and the NB shape.
static std::vector<std::pair<void*, size_t>> sweep_state(const gmf_sweep* s) {
    std::vector<std::pair<void*, size_t>> v;
    for (const gmf_model* h : s->models) {
        v.push_back({h->L, sizeof(float) * (size_t)h->n * h->KP});
        v.push_back({h->R, sizeof(float) * (size_t)h->m * h->KP});
        v.push_back({h->GbR, sizeof(float) * (size_t)h->n * h->fr});
        v.push_back({h->HbR, sizeof(float) * (size_t)h->n * h->fr});
        v.push_back({h->GbC, sizeof(float) * (size_t)h->m * h->fc});
        v.push_back({h->HbC, sizeof(float) * (size_t)h->m * h->fc});
        v.push_back({h->cntR, sizeof(int) * (size_t)h->n});
        v.push_back({h->cntC, sizeof(int) * (size_t)h->m});
        v.push_back({h->alpha, sizeof(float)});
    }
    return v;
}

static cudaError_t copy_state(const std::vector<std::pair<void*, size_t>>& st, char* save, bool to_save,
                              cudaStream_t stream) {
    size_t off = 0;
    for (const auto& b : st) {
        if (b.second) {
            const cudaError_t e = to_save ? cudaMemcpyAsync(save + off, b.first, b.second, cudaMemcpyDeviceToDevice, stream)
                                          : cudaMemcpyAsync(b.first, save + off, b.second, cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return e;
        }
        off += (b.second + 255) & ~(size_t)255;
    }
    return cudaSuccess;
}

extern "C" int gmf_sweep_autotune(gmf_sweep* s, const int32_t* sigma, int32_t n_sweeps, int32_t* group_out,
                                  float* ms_out, void* stream) {
    if (!s || !sigma) return gmf_fail(GMF_ERR_ARG, "gmf_sweep_autotune: NULL argument");
    gmf_model* h0 = s->models[0];
    const int nm = (int)s->models.size();
    if (n_sweeps < 1 || n_sweeps > h0->nsw) return gmf_fail(GMF_ERR_ARG, "gmf_sweep_autotune: n_sweeps outside [1, S]");
    std::vector<char> seen(h0->nsw, 0);
    for (int w = 0; w < h0->nsw; w++) {
        if (sigma[w] < 0 || sigma[w] >= h0->nsw || seen[sigma[w]])
            return gmf_fail(GMF_ERR_ARG, "gmf_sweep_autotune: sigma is not a permutation");
        seen[sigma[w]] = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (gmf_model* h : s->models) {
        const int rc = gmf_stage_schedule(h, sigma, 0, h->nsw, st);
        if (rc) return rc;
    }
    const auto state = sweep_state(s);
    size_t bytes = 0;
    for (const auto& b : state) bytes += (b.second + 255) & ~(size_t)255;
    char* save = nullptr;
    if (cudaMalloc(&save, bytes) != cudaSuccess) return gmf_fail(GMF_ERR_OOM, "gmf_sweep_autotune: no room for the state copy");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = copy_state(state, save, true, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // candidates: all models in one launch, then halved groups down to one model per launch
    std::vector<int> cand;
    for (int g = nm;; g = (g + 1) / 2) {
        cand.push_back(g);
        if (g == 1) break;
    }
    cand.push_back(GMF_SWEEP_SEQUENTIAL);  // and every model's own launches, model after model
    if (s->mixed) cand.push_back(GMF_SWEEP_PERSISTENT);  // and one persistent launch per sweep
    if (ms_out)
        for (int i = 0; i <= nm + 1; i++) ms_out[i] = -1.f;
    std::vector<int64_t> t_saved;
    for (gmf_model* h : s->models) t_saved.push_back(h->t);
    int inner_rc = GMF_OK;  // a failed single-model epoch (its message is kept)
    // one candidate's trial: its launches for sweeps [0, count) of every model
    auto trial = [&](int g, int count) -> cudaError_t {
        if (g != GMF_SWEEP_SEQUENTIAL) {
            cudaError_t r = g == GMF_SWEEP_PERSISTENT ? cudaMemsetAsync(s->gctr, 0, sizeof(unsigned), st) : cudaSuccess;
            for (int w = 0; w < count && r == cudaSuccess; w++) r = launch(s, w, st, g);
            return r;
        }
        for (int i = 0; i < nm; i++) {
            gmf_model* h = s->models[s->order[i]];
            const int rc = gmf_sgd_sweeps(h, sigma, 0, count, st);
            h->t = t_saved[(size_t)s->order[i]];
            if (rc) {
                inner_rc = rc;
                return cudaErrorUnknown;
            }
        }
        return cudaSuccess;
    };
    int best = nm;
    float best_ms = 0.f;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess; c++) {
        const int g = cand[c];
        // one untimed run (first use of this launch shape), then the timed run, each from the saved state
        e = trial(g, g == GMF_SWEEP_SEQUENTIAL ? n_sweeps : 1);
        if (e == cudaSuccess) e = copy_state(state, save, false, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = trial(g, n_sweeps);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = copy_state(state, save, false, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms_out) ms_out[g == GMF_SWEEP_SEQUENTIAL ? nm : g == GMF_SWEEP_PERSISTENT ? nm + 1 : g - 1] = ms;
        if (c == 0 || ms < best_ms) {
            best_ms = ms;
            best = g;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    for (int i = 0; i < nm; i++) s->models[i]->t = t_saved[(size_t)i];
    if (inner_rc != GMF_OK) return inner_rc;  // gmf_last_error holds the failing call's message
    if (e != cudaSuccess)
        return gmf_fail(GMF_ERR_CUDA, (std::string("gmf_sweep_autotune: ") + cudaGetErrorString(e)).c_str());
    const int rc = gmf_sweep_set_group(s, best == nm ? 0 : best);  // (the negative settings are kept as they are)
    if (rc) return rc;
    if (group_out) *group_out = best;
    return GMF_OK;
}

extern "C" gmf_model* gmf_sweep_model(gmf_sweep* s, int32_t i) {
    if (!s || i < 0 || i >= (int32_t)s->models.size()) return nullptr;
    return s->models[i];
}

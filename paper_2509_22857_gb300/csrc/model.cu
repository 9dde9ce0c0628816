// Compiled CNN programs: weight plaintexts resident in HBM, and a batched
// executor that runs every step for all images of a batch in the same
// kernels (so each evaluation key and each weight plaintext is read once per
// batch rather than once per image).
#include <algorithm>
#include <cstring>
#include <memory>
#include <map>
#include <set>

#include "host.h"

namespace {

struct MTensor {
    int n_ct, level;
    double scale;
};

struct MLinear {
    int level = 0;
    std::vector<int> baby_ct, baby_step;           // distinct (ct, b != 0)
    std::vector<int> g_out, g_giant, g_tb, g_te;   // groups
    std::vector<int> t_ct, t_baby;
    std::vector<u64 *> t_pt;                       // resident plaintext of each term
    std::vector<u64 *> bias_pt;                    // per output ct (nullable)
    // encoded on demand: the term rows stay sparse on the device
    bool on_demand = false;
    double w_scale = 0;
    int n_rows = 0;
    long long *d_begin = nullptr;
    int *d_slot = nullptr;
    double *d_val = nullptr;
    std::vector<int> t_vid;                        // row of each term
    // double hoisting: baby rotations stay in Q_l u P; plaintexts are
    // encoded over Q_l u P (the unrotated terms use their first l+1 limbs)
    bool dh = false;
};

struct MStep {
    int kind = 0, src = -1, src2 = -1, dst = -1;
    MLinear lin;
    u64 *c1 = nullptr, *c0 = nullptr, *cval = nullptr;   // per-limb residues
    u64 *c1v = nullptr, *c0v = nullptr;                   // ACT per channel: [n_ct] plaintexts
    std::vector<int> rot;
    int level = 0;
};

}  // namespace

struct fhe_model {
    fhe_ctx *ctx;
    std::vector<MTensor> tensors;
    std::vector<MStep> steps;
    std::vector<int> last_use;
    int input = 0, output = 0;
    std::vector<void *> owned;
    size_t pt_bytes = 0;
};

static int residues_of(fhe_model *m, double v, int level, u64 **out) {
    fhe_ctx *c = m->ctx;
    std::vector<u64> r(level + 1);
    for (int l = 0; l <= level; l++) r[l] = h_double_mod(v, c->primes[l]);
    void *d;
    FHE_TRY(dev_alloc(c, &d, r.size() * 8));
    m->owned.push_back(d);
    FHE_CU(cudaMemcpy(d, r.data(), r.size() * 8, cudaMemcpyHostToDevice));
    *out = (u64 *)d;
    return FHE_OK;
}

static int encode_vec(fhe_model *m, const double *vec, double scale, int level, u64 **out, bool ext = false) {
    fhe_ctx *c = m->ctx;
    std::vector<double> coef(c->N);
    c->enc.encode(vec, nullptr, (size_t)c->N / 2, scale, coef.data());
    void *d;
    const size_t bytes = (size_t)(level + 1 + (ext ? c->alpha : 0)) * c->N * 8;
    FHE_TRY(dev_alloc(c, &d, bytes));
    m->owned.push_back(d);
    m->pt_bytes += bytes;
    FHE_TRY(op_encode_to(c, coef.data(), level, (u64 *)d, 0, ext));
    *out = (u64 *)d;
    return FHE_OK;
}

// per-channel activation coefficients: each ciphertext's two slot vectors
// encoded at their scales and the tensor's level, contiguous per set
static int encode_act_vecs(fhe_model *m, const fhe_step_desc &sd, const MTensor &ti, MStep *st) {
    fhe_ctx *c = m->ctx;
    const size_t ns = (size_t)c->N / 2;
    const long long P = (long long)(ti.level + 1) * c->N;
    for (int set = 0; set < 2; set++) {
        void *d;
        FHE_TRY(dev_alloc(c, &d, (size_t)ti.n_ct * P * 8));
        m->owned.push_back(d);
        const double *vecs = set ? sd.act_c0_vecs : sd.act_c1_vecs;
        const double scale = set ? sd.act_c0_scale : sd.act_c1_scale;
        std::vector<double> coef(c->N);
        for (int k = 0; k < ti.n_ct; k++) {
            c->enc.encode(vecs + (size_t)k * ns, nullptr, ns, scale, coef.data());
            FHE_TRY(op_encode_to(c, coef.data(), ti.level, (u64 *)d + k * P, 0));
        }
        (set ? st->c0v : st->c1v) = (u64 *)d;
    }
    return FHE_OK;
}

// inverse of an odd a modulo m = 2^k (Newton: each step doubles the correct
// low bits; a * a = 1 mod 8 starts with three)
static int inverse_mod_2n(int a, long long m) {
    unsigned long long x = (unsigned long long)a, ua = (unsigned long long)a;
    for (int i = 0; i < 6; i++) x = x * (2ull - ua * x);
    return (int)(x & (unsigned long long)(m - 1));
}

static int load_linear(fhe_model *m, const fhe_step_desc &sd, MStep &st) {
    fhe_ctx *c = m->ctx;
    MLinear &L = st.lin;
    const MTensor &tin = m->tensors[st.src], &tout = m->tensors[st.dst];
    L.level = tin.level;
    L.dh = sd.double_hoist != 0;
    if (tout.level != tin.level) return fhe_fail(FHE_E_LEVEL, "linear step changes level");
    const size_t ns = (size_t)c->N / 2;
    if (sd.n_groups < 0 || (sd.n_groups > 0 && (!sd.group_out || !sd.group_giant || !sd.group_term_begin)))
        return fhe_fail(FHE_E_INVAL, "linear step: missing group arrays");
    const int n_terms = sd.n_groups > 0 ? sd.group_term_begin[sd.n_groups] : 0;
    if (n_terms > 0 && (!sd.term_ct || !sd.term_baby || !sd.term_vec_id || (!sd.vecs && !sd.sparse_vec_begin) ||
                        sd.n_vecs < 1))
        return fhe_fail(FHE_E_INVAL, "linear step: missing term arrays");
    // every distinct vector is encoded once; its terms share the plaintext
    std::vector<u64 *> vec_pt(n_terms > 0 ? sd.n_vecs : 0, nullptr);
    std::set<std::pair<int, int>> baby;
    std::vector<int> has_zero(tout.n_ct, 0);
    for (int g = 0; g < sd.n_groups; g++) {
        const int o = sd.group_out[g];
        if (o < 0 || o >= tout.n_ct) return fhe_fail(FHE_E_INVAL, "linear step: output index");
        if (sd.group_giant[g] == 0) has_zero[o] = 1;
        L.g_out.push_back(o);
        L.g_giant.push_back(sd.group_giant[g]);
        L.g_tb.push_back(sd.group_term_begin[g]);
        L.g_te.push_back(sd.group_term_begin[g + 1]);
        if (sd.group_term_begin[g + 1] < sd.group_term_begin[g]) return fhe_fail(FHE_E_INVAL, "term ranges");
    }
    for (int o = 0; o < tout.n_ct; o++)
        if (!has_zero[o]) {
            L.g_out.push_back(o);
            L.g_giant.push_back(0);
            L.g_tb.push_back(n_terms);
            L.g_te.push_back(n_terms);
        }
    if (n_terms > 0 && sd.sparse_vec_begin) {
        // encoded on demand: rows checked and copied to the device as given
        const int64_t *bg = sd.sparse_vec_begin;
        if (!sd.sparse_slot || !sd.sparse_val || bg[0] != 0)
            return fhe_fail(FHE_E_INVAL, "linear step: sparse rows");
        for (int v = 0; v < sd.n_vecs; v++)
            if (bg[v + 1] < bg[v]) return fhe_fail(FHE_E_INVAL, "linear step: sparse row offsets");
        const long long nnz = bg[sd.n_vecs];
        for (long long e = 0; e < nnz; e++)
            if (sd.sparse_slot[e] < 0 || (size_t)sd.sparse_slot[e] >= ns)
                return fhe_fail(FHE_E_INVAL, "linear step: sparse slot index");
        const EncTab *et;
        FHE_TRY(enc_tables(c, &et));
        void *d;
        FHE_TRY(dev_alloc(c, &d, (size_t)(sd.n_vecs + 1) * 8));
        m->owned.push_back(d);
        FHE_CU(cudaMemcpy(d, bg, (size_t)(sd.n_vecs + 1) * 8, cudaMemcpyHostToDevice));
        L.d_begin = (long long *)d;
        FHE_TRY(dev_alloc(c, &d, (size_t)nnz * 4));
        m->owned.push_back(d);
        FHE_CU(cudaMemcpy(d, sd.sparse_slot, (size_t)nnz * 4, cudaMemcpyHostToDevice));
        L.d_slot = (int *)d;
        FHE_TRY(dev_alloc(c, &d, (size_t)nnz * 8));
        m->owned.push_back(d);
        FHE_CU(cudaMemcpy(d, sd.sparse_val, (size_t)nnz * 8, cudaMemcpyHostToDevice));
        L.d_val = (double *)d;
        L.on_demand = true;
        L.w_scale = sd.w_scale;
        L.n_rows = sd.n_vecs;
    }
    for (int t = 0; t < n_terms; t++) {
        const int ct = sd.term_ct[t], b = sd.term_baby[t];
        if (ct < 0 || ct >= tin.n_ct) return fhe_fail(FHE_E_INVAL, "linear step: input index");
        L.t_ct.push_back(ct);
        L.t_baby.push_back(b);
        if (galois_of_step(c, b) != 1) baby.insert({ct, b});
        const int v = sd.term_vec_id[t];
        if (v < 0 || v >= sd.n_vecs) return fhe_fail(FHE_E_INVAL, "linear step: vector index");
        L.t_vid.push_back(v);
        if (L.on_demand) {
            L.t_pt.push_back(nullptr);
            continue;
        }
        if (!vec_pt[v]) FHE_TRY(encode_vec(m, sd.vecs + (size_t)v * ns, sd.w_scale, L.level, &vec_pt[v], L.dh));
        L.t_pt.push_back(vec_pt[v]);
    }
    for (auto &p : baby) {
        L.baby_ct.push_back(p.first);
        L.baby_step.push_back(p.second);
    }
    L.bias_pt.assign(tout.n_ct, nullptr);
    for (int b = 0; b < sd.n_bias; b++) {
        const int o = sd.bias_out[b];
        if (o < 0 || o >= tout.n_ct) return fhe_fail(FHE_E_INVAL, "bias index");
        FHE_TRY(encode_vec(m, sd.bias_vec + (size_t)b * ns, sd.bias_scale, L.level, &L.bias_pt[o]));
    }
    return FHE_OK;
}

extern "C" int fhe_model_load(fhe_ctx *c, const fhe_model_desc *d, fhe_model **out) {
    if (!c || !d || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (d->n_tensors <= 0 || !d->tensor_n_ct || !d->tensor_level || !d->tensor_scale)
        return fhe_fail(FHE_E_INVAL, "model without tensors");
    FHE_CU(cudaSetDevice(c->dev));
    std::unique_ptr<fhe_model> m(new fhe_model());
    m->ctx = c;
    for (int t = 0; t < d->n_tensors; t++) {
        if (d->tensor_level[t] < 0 || d->tensor_level[t] > c->L) return fhe_fail(FHE_E_LEVEL, "tensor level");
        if (d->tensor_n_ct[t] <= 0) return fhe_fail(FHE_E_INVAL, "tensor size");
        m->tensors.push_back({d->tensor_n_ct[t], d->tensor_level[t], d->tensor_scale[t]});
    }
    if (d->input_tensor < 0 || d->input_tensor >= d->n_tensors || d->output_tensor < 0 ||
        d->output_tensor >= d->n_tensors)
        return fhe_fail(FHE_E_INVAL, "input / output tensor");
    m->input = d->input_tensor;
    m->output = d->output_tensor;
    auto check_t = [&](int t) { return t >= 0 && t < d->n_tensors; };
    int rc = FHE_OK;
    for (int i = 0; i < d->n_steps && rc == FHE_OK; i++) {
        const fhe_step_desc &sd = d->steps[i];
        MStep st;
        st.kind = sd.kind;
        st.src = sd.src;
        st.src2 = sd.src2;
        st.dst = sd.dst;
        if (!check_t(sd.src) || !check_t(sd.dst) || (sd.kind == FHE_STEP_ADD && !check_t(sd.src2))) {
            rc = fhe_fail(FHE_E_INVAL, "step " + std::to_string(i) + ": tensor index");
            break;
        }
        const MTensor &ti = m->tensors[sd.src], &to = m->tensors[sd.dst];
        switch (sd.kind) {
        case FHE_STEP_LINEAR:
            rc = load_linear(m.get(), sd, st);
            break;
        case FHE_STEP_RESCALE:
            if (to.level != ti.level - 1 || ti.level < 1 || to.n_ct != ti.n_ct)
                rc = fhe_fail(FHE_E_LEVEL, "rescale step levels");
            break;
        case FHE_STEP_ACT:
            if (to.level != ti.level || to.n_ct != ti.n_ct) rc = fhe_fail(FHE_E_LEVEL, "act step levels");
            if (rc == FHE_OK) rc = residues_of(m.get(), sd.c1, ti.level, &st.c1);
            if (rc == FHE_OK) rc = residues_of(m.get(), sd.c0, ti.level, &st.c0);
            if (rc == FHE_OK && (sd.act_c1_vecs != nullptr) != (sd.act_c0_vecs != nullptr))
                rc = fhe_fail(FHE_E_INVAL, "act step: both per-channel vector sets or neither");
            if (rc == FHE_OK && sd.act_c1_vecs) rc = encode_act_vecs(m.get(), sd, ti, &st);
            break;
        case FHE_STEP_CMUL:
            if (to.level != ti.level || to.n_ct != ti.n_ct) rc = fhe_fail(FHE_E_LEVEL, "cmul step levels");
            if (rc == FHE_OK) rc = residues_of(m.get(), sd.value, ti.level, &st.cval);
            break;
        case FHE_STEP_ROTSUM:
            if (to.level != ti.level || to.n_ct != ti.n_ct) rc = fhe_fail(FHE_E_LEVEL, "rotsum step levels");
            for (int k = 0; k < sd.n_steps; k++) st.rot.push_back(sd.steps[k]);
            break;
        case FHE_STEP_DROP:
            if (to.level != sd.level || sd.level > ti.level || to.n_ct != ti.n_ct)
                rc = fhe_fail(FHE_E_LEVEL, "drop step levels");
            st.level = sd.level;
            break;
        case FHE_STEP_ADD: {
            const MTensor &t2 = m->tensors[sd.src2];
            if (t2.level != ti.level || to.level != ti.level || t2.n_ct != ti.n_ct || to.n_ct != ti.n_ct)
                rc = fhe_fail(FHE_E_LEVEL, "add step levels");
            break;
        }
        default:
            rc = fhe_fail(FHE_E_INVAL, "unknown step kind");
        }
        m->steps.push_back(std::move(st));
    }
    if (rc != FHE_OK) {
        cudaDeviceSynchronize();
        for (void *p : m->owned) dev_free(p);
        return rc;
    }
    m->last_use.assign(m->tensors.size(), -1);
    for (int i = 0; i < (int)m->steps.size(); i++) {
        m->last_use[m->steps[i].src] = i;
        if (m->steps[i].src2 >= 0) m->last_use[m->steps[i].src2] = i;
    }
    FHE_CU(cudaDeviceSynchronize());
    *out = m.release();
    return FHE_OK;
}

extern "C" int fhe_model_free(fhe_model *m) {
    if (!m) return FHE_OK;
    cudaDeviceSynchronize();
    for (void *p : m->owned) dev_free(p);
    delete m;
    return FHE_OK;
}

// ================================================================ executor

namespace {

// Buffers that persist across executions (pipeline mode): every temporary of
// a step and every device work list is allocated on first use and reused, so
// later executions of the same steps issue kernels only (and can be captured
// in a CUDA graph).
struct Persist {
    std::map<std::pair<int, int>, u64 *> tmp;      // (step, index) -> device buffer
    std::map<std::pair<int, long long>, char *> lists;   // (variant, step and sub-list) -> device work list
    std::vector<void *> owned;
    int variant = 0;                               // which set of work lists (pipeline parity)
    u64 *ks_ws = nullptr;                          // this executor's key-switch workspace
    u64 *rs_ws = nullptr;                          // and rescale workspace

    ~Persist() {
        for (void *p : owned) cudaFree(p);
    }
};

struct Exec {
    fhe_model *m;
    const fhe_evk *evk;
    int B;
    cudaStream_t s;
    std::vector<u64 *> buf;               // per tensor: [B][n_ct][2][level+1][N]
    std::vector<std::vector<char>> host_stage;
    Persist *pers = nullptr;              // non-null: pipeline mode
    int cur_step = -1;
    long long list_sub = 0;               // which work list of the current step
    // optional timing: events bracketing each phase, summed per phase kind
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> *prof = nullptr;
    void mark(int kind, bool begin) {
        if (!prof) return;
        if (begin) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
            prof->push_back({kind, {a, b}});
        } else {
            cudaEventRecord(prof->back().second.second, s);
        }
    }

    long long ctst(int t) const { return 2ll * (m->tensors[t].level + 1) * m->ctx->N; }
    long long item(int t) const { return (long long)m->tensors[t].n_ct * ctst(t); }

    int alloc_t(int t) {
        if (buf[t]) return FHE_OK;
        if (pers) return fhe_fail(FHE_E_INVAL, "internal: tensor without a buffer in pipeline mode");
        const size_t bytes = (size_t)B * item(t) * 8;
        FHE_ALLOC_ASYNC(&buf[t], bytes, s);
        return FHE_OK;
    }
    void release(int t) {
        if (pers) return;
        if (buf[t] && t != m->output) {
            cudaFreeAsync(buf[t], s);
            buf[t] = nullptr;
        }
    }
    // a temporary of the current step (index idx): stream-ordered, or persistent
    int tmp(int idx, size_t bytes, u64 **out) {
        if (!pers) {
            FHE_ALLOC_ASYNC(out, bytes, s);
            return FHE_OK;
        }
        auto key = std::make_pair(cur_step, idx);
        auto it = pers->tmp.find(key);
        if (it == pers->tmp.end()) {
            void *p;
            FHE_TRY(dev_alloc(m->ctx, &p, bytes));
            pers->owned.push_back(p);
            it = pers->tmp.emplace(key, (u64 *)p).first;
        }
        *out = it->second;
        return FHE_OK;
    }
    void tmp_free(void *p) {
        if (!pers && p) cudaFreeAsync(p, s);
    }
    // a work list in device memory with the given host content
    int work_list(const char *host, size_t bytes, char **out) {
        if (!pers) {
            host_stage.emplace_back(host, host + bytes);
            FHE_ALLOC_ASYNC(out, bytes + 16, s);
            FHE_CU(cudaMemcpyAsync(*out, host_stage.back().data(), bytes, cudaMemcpyHostToDevice, s));
            return FHE_OK;
        }
        auto key = std::make_pair(pers->variant, ((long long)cur_step << 40) + list_sub);
        auto it = pers->lists.find(key);
        if (it == pers->lists.end()) {
            // Lists are made by the eager ticks that precede any capture.  The
            // upload is ordered on this executor's own stream (non-blocking):
            // a plain cudaMemcpy from pageable memory runs on the legacy
            // stream and may return before its DMA lands, so a kernel on
            // this stream could read a partly written list.
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            FHE_CU(cudaStreamIsCapturing(s, &cs));
            if (cs != cudaStreamCaptureStatusNone)
                return fhe_fail(FHE_E_INVAL, "internal: work list first needed inside a graph capture");
            void *p;
            FHE_TRY(dev_alloc(m->ctx, &p, bytes + 16));
            pers->owned.push_back(p);
            FHE_CU(cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, s));
            FHE_CU(cudaStreamSynchronize(s));
            it = pers->lists.emplace(key, (char *)p).first;
        }
        *out = it->second;
        return FHE_OK;
    }
    const u64 *key_for(int step, int *err) {
        const int k = galois_of_step(m->ctx, step);
        auto it = evk->galois.find(k);
        if (it == evk->galois.end()) {
            *err = fhe_fail(FHE_E_NOKEY, "no Galois key for rotation step " + std::to_string(step));
            return nullptr;
        }
        *err = FHE_OK;
        return it->second;
    }
    // A whole key switch of many items runs in launches of at most the
    // context's ks_item_cap items (its workspace is then sized for the cap);
    // the phases of a split key switch carry state and run whole.
    int keyswitch(const KsArgs &a, int phases = KS_ALL) {
        const int cap = m->ctx->ks_item_cap;
        if (phases != KS_ALL || cap <= 0 || a.n_items <= cap)
            return op_keyswitch(m->ctx, a, s, pers ? pers->ks_ws : nullptr, phases);
        for (int i0 = 0; i0 < a.n_items; i0 += cap) {
            KsArgs b = a;
            b.n_items = std::min(cap, a.n_items - i0);
            b.d = a.d + (long long)i0 * a.d_item;
            if (a.add0) b.add0 = a.add0 + (long long)i0 * a.add_item;
            if (a.add1) b.add1 = a.add1 + (long long)i0 * a.add_item;
            if (a.base) b.base = a.base + (long long)i0 * a.base_item;
            b.out = a.out + (long long)i0 * a.out_item;
            FHE_TRY(op_keyswitch(m->ctx, b, s, pers ? pers->ks_ws : nullptr, phases));
        }
        return FHE_OK;
    }

    int ip_babies(const KsArgs &a, const IpBabies &bb) {
        return op_ks_ip_babies(m->ctx, a, bb, s, pers ? pers->ks_ws : nullptr);
    }

    // out = base + rot(x, step) for n items of one tensor-like layout
    int rotate_items(const u64 *x, long long x_item, int step, const u64 *base, long long base_item, u64 *out,
                     long long out_item, int n, int level) {
        int err;
        const u64 *key = key_for(step, &err);
        if (!key) return err;
        KsArgs a;
        memset(&a, 0, sizeof(a));
        const long long nlN = (long long)(level + 1) * m->ctx->N;
        a.d = x + nlN;
        a.d_item = x_item;
        a.galois = galois_of_step(m->ctx, step);
        a.key = key;
        a.key_digits_top = evk->digits;
        a.add0 = x;
        a.add_item = x_item;
        a.base = base;
        a.base_item = base_item;
        a.out = out;
        a.out_item = out_item;
        a.n_items = n;
        a.level = level;
        return keyswitch(a);
    }

    // Input chunks of a linear step: consecutive input ciphertexts whose
    // baby-step rotations (B images each) fit LIN_CHUNK_BYTES and whose
    // sources number at most the context's lin_chunk_srcs, so that the
    // source tiles a MAC CTA reads stay in L1 across the output groups.  A
    // step whose inputs all fit is one chunk; chunking changes no result.
    static constexpr size_t LIN_CHUNK_BYTES = 32ull << 30;

    int linear(const MStep &st) {
        const MLinear &L = st.lin;
        fhe_ctx *c = m->ctx;
        const int lv = L.level;
        const long long cs = ctst(st.src);
        const u64 *in = buf[st.src];
        u64 *out = buf[st.dst];
        const long long in_item = item(st.src), out_item = item(st.dst);
        const int n_in = m->tensors[st.src].n_ct;
        const long long nlN = (long long)(lv + 1) * c->N;
        // double hoisting: a baby rotation, a rotated term's plaintext and a
        // group's sum of rotated terms live in Q_l u P
        const long long extN = (long long)(lv + 1 + c->alpha) * c->N;
        const long long rcs = L.dh ? 2 * extN : cs;   // words of one rotated copy
        const long long pt_limbs = L.dh ? extN : nlN;  // words of one plaintext
        // babies of each input, then the chunks
        std::vector<int> nb(n_in, 0), first_baby(n_in + 1, 0);
        for (size_t k = 0; k < L.baby_ct.size(); k++) nb[L.baby_ct[k]]++;
        for (int ct = 0; ct < n_in; ct++) first_baby[ct + 1] = first_baby[ct] + nb[ct];
        const size_t baby_bytes = (size_t)B * rcs * 8;
        std::vector<int> cut{0};
        int max_babies = 0;
        {
            int b = 0, srcs = 0;
            for (int ct = 0; ct < n_in; ct++) {
                const bool full = ct > cut.back() &&
                                  ((size_t)(b + nb[ct]) * baby_bytes > LIN_CHUNK_BYTES ||
                                   srcs + nb[ct] + 1 > m->ctx->lin_chunk_srcs);
                if (full) {
                    max_babies = std::max(max_babies, b);
                    cut.push_back(ct);
                    b = 0;
                    srcs = 0;
                }
                b += nb[ct];
                srcs += nb[ct] + 1;
            }
            max_babies = std::max(max_babies, b);
            cut.push_back(n_in);
        }
        int ti = 0;
        std::vector<u64 *> rb(max_babies, nullptr);
        for (int k = 0; k < max_babies; k++) FHE_TRY(tmp(ti++, baby_bytes, &rb[k]));
        // accumulators of the giant steps (g != 0); g == 0 goes straight to out
        const int ng = (int)L.g_out.size();
        std::vector<u64 *> acc(ng, nullptr);
        for (int g = 0; g < ng; g++)
            if (galois_of_step(c, L.g_giant[g]) != 1) FHE_TRY(tmp(ti++, (size_t)B * cs * 8, &acc[g]));
        // double hoisting: each group's sum of rotated terms over Q_l u P,
        // for the groups that have rotated terms; written[g] tracks whether
        // a MAC has written it yet (later pieces accumulate)
        std::vector<u64 *> ext_sum(ng, nullptr);
        std::vector<char> ext_written(ng, 0);
        if (L.dh)
            for (int g = 0; g < ng; g++)
                for (int t = L.g_tb[g]; t < L.g_te[g]; t++)
                    if (galois_of_step(c, L.t_baby[t]) != 1) {
                        FHE_TRY(tmp(ti++, (size_t)B * 2 * extN * 8, &ext_sum[g]));
                        break;
                    }
        // scratch of the plaintexts encoded on demand: rows of one batch of
        // groups (FFT buffer N doubles + (lv+1) limbs per row, at most the
        // context's on_demand_bytes)
        int od_rows = 0;
        double *od_buf = nullptr;
        u64 *od_pt = nullptr;
        const EncTab *enc = nullptr;
        if (L.on_demand) {
            FHE_TRY(enc_tables(c, &enc));
            const size_t per_row = (size_t)(pt_limbs + c->N) * 8;
            od_rows = (int)std::min<size_t>((size_t)L.n_rows, std::max<size_t>(1, c->on_demand_bytes / per_row));
            od_rows = std::min(od_rows, 65535);
            FHE_TRY(tmp(ti++, (size_t)od_rows * c->N * 8, (u64 **)&od_buf));
            FHE_TRY(tmp(ti++, (size_t)od_rows * pt_limbs * 8, &od_pt));
        }
        for (size_t ch = 0; ch + 1 < cut.size(); ch++) {
            const int lo = cut[ch], hi = cut[ch + 1];
            // baby-step rotations of this chunk's inputs: the rotations of one
            // input share its ModUp (hoisting); each then needs an inner
            // product and a ModDown
            mark(10, true);
            for (int ct = lo; ct < hi; ct++) {
                if (!nb[ct]) continue;
                const u64 *x = in + ct * cs;
                KsArgs a;
                memset(&a, 0, sizeof(a));
                a.d = x + nlN;
                a.d_item = in_item;
                a.galois = 1;
                a.n_items = B;
                a.level = lv;
                FHE_TRY(keyswitch(a, KS_MODUP));
                if (L.dh && c->lt[lv].n_digits <= 7) {
                    // double hoisting: the input's rotations in batches, each
                    // batch one pass over the ModUp digits and c0
                    for (int k0 = first_baby[ct]; k0 < first_baby[ct + 1]; k0 += KS_BABIES_MAX) {
                        IpBabies bb;
                        memset(&bb, 0, sizeof(bb));
                        for (int kk = k0; kk < std::min(k0 + KS_BABIES_MAX, first_baby[ct + 1]); kk++) {
                            int err;
                            const u64 *key = key_for(L.baby_step[kk], &err);
                            if (!key) return err;
                            bb.key[bb.n] = key;
                            bb.out[bb.n] = rb[kk - first_baby[lo]];
                            bb.gal_inv[bb.n] = inverse_mod_2n(galois_of_step(c, L.baby_step[kk]), 2 * c->N);
                            bb.n++;
                        }
                        KsArgs b = a;
                        b.ip_fold = x;
                        b.ip_fold_item = in_item;
                        b.ip_out_item = rcs;
                        FHE_TRY(ip_babies(b, bb));
                    }
                    continue;
                }
                for (int kk = first_baby[ct]; kk < first_baby[ct + 1]; kk++) {
                    int err;
                    const u64 *key = key_for(L.baby_step[kk], &err);
                    if (!key) return err;
                    const int gal = galois_of_step(c, L.baby_step[kk]);
                    a.key = key;
                    a.key_digits_top = evk->digits;
                    a.ip_galois = gal;
                    if (L.dh) {
                        // the rotation stays in Q_l u P: inner product plus
                        // P sigma(c0), no ModDown
                        a.ip_out = rb[kk - first_baby[lo]];
                        a.ip_out_item = rcs;
                        a.ip_fold = x;
                        a.ip_fold_item = in_item;
                        FHE_TRY(keyswitch(a, KS_IP));
                        continue;
                    }
                    a.add0 = x;
                    a.add_item = in_item;
                    a.add_galois = gal;
                    a.out = rb[kk - first_baby[lo]];
                    a.out_item = cs;
                    FHE_TRY(keyswitch(a, KS_IP | KS_MODDOWN));
                }
            }
            mark(10, false);
            // sources: the input ciphertexts, then this chunk's baby-step rotations
            // (double hoisting: the rotations are the sources of a second
            // MAC over Q_l u P, numbered from 0)
            std::vector<MacSrc> hs, hs_ext;
            for (int ct = 0; ct < n_in; ct++) hs.push_back(MacSrc{in + ct * cs, in_item});
            for (int kk = first_baby[lo]; kk < first_baby[hi]; kk++)
                (L.dh ? hs_ext : hs).push_back(MacSrc{rb[kk - first_baby[lo]], rcs});
            auto src_of = [&](int ct, int b) -> int {
                if (galois_of_step(c, b) == 1) return ct;
                for (int kk = first_baby[ct]; kk < first_baby[ct + 1]; kk++)
                    if (L.baby_step[kk] == b) return (L.dh ? 0 : n_in) + (kk - first_baby[lo]);
                return -1;
            };
            // the groups of this chunk with their term ranges
            struct CG {
                int g, tb, tc;
            };
            std::vector<CG> cg;
            for (int g = 0; g < ng; g++) {
                // the group's terms of this chunk (terms are ordered by input ct)
                int tb = L.g_tb[g], te = L.g_te[g];
                while (tb < te && L.t_ct[tb] < lo) tb++;
                int tc = tb;
                while (tc < te && L.t_ct[tc] < hi) tc++;
                if (ch > 0 && tc == tb) continue;
                cg.push_back(CG{g, tb, tc});
            }
            // pieces of groups (term ranges), batched: all at once, or
            // (plaintexts encoded on demand) as many as keep their distinct
            // rows within the encoding scratch; a group may end one batch and
            // continue in the next (its later pieces accumulate)
            struct Piece {
                int g, tb, tc;
                bool cont;
            };
            std::vector<std::vector<Piece>> batches(1);
            std::vector<std::vector<int>> batch_rows(1);
            {
                std::map<int, int> seen;
                for (const CG &x : cg) {
                    int t0 = x.tb;
                    bool cont = false;
                    if (!L.on_demand || x.tb == x.tc) {
                        batches.back().push_back(Piece{x.g, x.tb, x.tc, false});
                        continue;
                    }
                    for (int t = x.tb; t < x.tc; t++) {
                        const int v = L.t_vid[t];
                        if (seen.count(v)) continue;
                        if ((int)seen.size() == od_rows) {
                            if (t > t0) {
                                batches.back().push_back(Piece{x.g, t0, t, cont});
                                cont = true;
                                t0 = t;
                            }
                            batches.emplace_back();
                            batch_rows.emplace_back();
                            seen.clear();
                        }
                        seen[v] = (int)batch_rows.back().size();
                        batch_rows.back().push_back(v);
                    }
                    batches.back().push_back(Piece{x.g, t0, x.tc, cont});
                }
            }
            for (size_t bi = 0; bi < batches.size(); bi++) {
                const std::vector<Piece> &pcs = batches[bi];
                const std::vector<int> &rows = batch_rows[bi];
                std::map<int, int> row_slot;
                for (size_t k = 0; k < rows.size(); k++) row_slot[rows[k]] = (int)k;
                if (L.on_demand && !rows.empty()) {
                    // encode this batch's rows
                    char *dv;
                    list_sub = ((long long)ch << 20) + 2 * (long long)bi + 1;
                    FHE_TRY(work_list((const char *)rows.data(), rows.size() * sizeof(int), &dv));
                    list_sub = 0;
                    mark(13, true);
                    FHE_CU(launch_encode_sparse(c->dc, *enc, (int)rows.size(), (const int *)dv, L.d_begin, L.d_slot,
                                                L.d_val, L.w_scale, lv, od_buf, od_pt, s, L.dh));
                    mark(13, false);
                    if (!pers) cudaFreeAsync(dv, s);
                }
                // grouped accumulation: the group's terms that share a
                // plaintext become one run (sources summed, one product);
                // the sum mod q does not depend on the order of the terms
                auto close_group = [](std::vector<MacTerm> &ht, MacGroup &G) {
                    std::stable_sort(ht.begin() + G.term_begin, ht.end(),
                                     [](const MacTerm &x, const MacTerm &y) { return x.pt < y.pt; });
                    for (int t = G.term_begin; t < (int)ht.size();) {
                        int e = t + 1;
                        while (e < (int)ht.size() && ht[e].pt == ht[t].pt) {
                            ht[e].run = 0;
                            e++;
                        }
                        ht[t].run = e - t;
                        t = e;
                    }
                    G.term_end = (int)ht.size();
                };
                // one MAC launch over its own work list (groups, terms, sources)
                auto run_mac = [&](const std::vector<MacGroup> &hg, const std::vector<MacTerm> &ht,
                                   const std::vector<MacSrc> &src, int ext, long long sub) -> int {
                    if (hg.empty()) return FHE_OK;
                    const size_t gb = hg.size() * sizeof(MacGroup), tb_ = ht.size() * sizeof(MacTerm),
                                 sb = src.size() * sizeof(MacSrc);
                    std::vector<char> lst(gb + tb_ + sb);
                    memcpy(lst.data(), hg.data(), gb);
                    if (tb_) memcpy(lst.data() + gb, ht.data(), tb_);
                    if (sb) memcpy(lst.data() + gb + tb_, src.data(), sb);
                    char *dw;
                    list_sub = sub;
                    FHE_TRY(work_list(lst.data(), lst.size(), &dw));
                    list_sub = 0;
                    MacArgs ma;
                    ma.groups = (const MacGroup *)dw;
                    ma.terms = (const MacTerm *)(dw + gb);
                    ma.srcs = (const MacSrc *)(dw + gb + tb_);
                    ma.n_groups = (int)hg.size();
                    ma.n_srcs = (int)src.size();
                    ma.n_items = B;
                    ma.level = lv;
                    ma.images_per_cta = c->mac_images;
                    ma.ext = ext;
                    mark(11, true);
                    FHE_CU(launch_mac(c->dc, ma, s));
                    mark(11, false);
                    if (!pers) cudaFreeAsync(dw, s);
                    return FHE_OK;
                };
                std::vector<MacGroup> hg, hg_ext;
                std::vector<MacTerm> ht, ht_ext;
                for (const Piece &pc : pcs) {
                    const int g = pc.g, tb = pc.tb, tc = pc.tc;
                    const int o = L.g_out[g];
                    MacGroup G;
                    if (!acc[g]) {
                        G.out = out + o * cs;
                        G.out_item = out_item;
                        G.bias = (ch == 0 && !pc.cont) ? L.bias_pt[o] : nullptr;
                    } else {
                        G.out = acc[g];
                        G.out_item = cs;
                        G.bias = nullptr;
                    }
                    G.accumulate = (ch > 0 || pc.cont) ? 1 : 0;
                    G.term_begin = (int)ht.size();
                    // double hoisting: the rotated terms form this group's
                    // piece of the MAC over Q_l u P
                    MacGroup GX;
                    GX.out = ext_sum[g];
                    GX.out_item = 2 * extN;
                    GX.bias = nullptr;
                    GX.accumulate = ext_written[g];
                    GX.term_begin = (int)ht_ext.size();
                    for (int t = tb; t < tc; t++) {
                        MacTerm T;
                        T.src = src_of(L.t_ct[t], L.t_baby[t]);
                        T.run = 1;
                        if (T.src < 0) return fhe_fail(FHE_E_INVAL, "internal: missing baby rotation");
                        T.pt = L.on_demand ? od_pt + (long long)row_slot[L.t_vid[t]] * pt_limbs : L.t_pt[t];
                        (L.dh && galois_of_step(c, L.t_baby[t]) != 1 ? ht_ext : ht).push_back(T);
                    }
                    close_group(ht, G);
                    hg.push_back(G);
                    if ((int)ht_ext.size() > GX.term_begin) {
                        close_group(ht_ext, GX);
                        hg_ext.push_back(GX);
                        ext_written[g] = 1;
                    }
                }
                FHE_TRY(run_mac(hg, ht, hs, 0, ((long long)ch << 20) + 2 * (long long)bi));
                FHE_TRY(run_mac(hg_ext, ht_ext, hs_ext, 1, ((long long)ch << 20) + (1ll << 19) + 2 * (long long)bi));
            }
        }
        // double hoisting: one ModDown per group of its rotated terms' sum,
        // added to the group's unrotated terms and bias
        if (L.dh) {
            mark(10, true);
            for (int g = 0; g < ng; g++) {
                if (!ext_written[g]) continue;
                u64 *dst = acc[g] ? acc[g] : out + L.g_out[g] * cs;
                const long long dst_item = acc[g] ? cs : out_item;
                KsArgs a;
                memset(&a, 0, sizeof(a));
                a.md_in = ext_sum[g];
                a.md_in_item = 2 * extN;
                a.base = dst;
                a.base_item = dst_item;
                a.out = dst;
                a.out_item = dst_item;
                a.n_items = B;
                a.level = lv;
                FHE_TRY(keyswitch(a, KS_MODDOWN));
            }
            mark(10, false);
        }
        mark(12, true);
        // giant steps: out_o += sum_g rot(acc_{o,g}, g) with one ModDown per
        // output: each term's ModUp and inner product accumulate in the
        // extended basis, the rotated c0 parts over Q
        u64 *c0acc = nullptr;
        for (int o = 0; o < m->tensors[st.dst].n_ct; o++) {
            bool first = true;
            KsArgs a;
            memset(&a, 0, sizeof(a));
            for (int g = 0; g < ng; g++) {
                if (!acc[g] || L.g_out[g] != o) continue;
                if (!c0acc) FHE_TRY(tmp(ti++, (size_t)B * nlN * 8, &c0acc));
                int err;
                const u64 *key = key_for(L.g_giant[g], &err);
                if (!key) return err;
                const int gal = galois_of_step(c, L.g_giant[g]);
                memset(&a, 0, sizeof(a));
                a.d = acc[g] + nlN;
                a.d_item = cs;
                a.galois = 1;
                a.key = key;
                a.key_digits_top = evk->digits;
                a.ip_galois = gal;
                a.ip_accumulate = first ? 0 : 1;
                a.n_items = B;
                a.level = lv;
                FHE_TRY(keyswitch(a, KS_MODUP | KS_IP));
                FHE_CU(launch_gather_acc(c->dc, acc[g], cs, c0acc, nlN, B, lv, gal, first ? 0 : 1, s));
                first = false;
            }
            if (first) continue;   // no giant step for this output
            u64 *op = out + o * cs;
            a.add0 = c0acc;
            a.add_item = nlN;
            a.add_galois = 1;
            a.base = op;
            a.base_item = out_item;
            a.out = op;
            a.out_item = out_item;
            FHE_TRY(keyswitch(a, KS_MODDOWN));
        }
        tmp_free(c0acc);
        mark(12, false);
        for (auto p : rb) tmp_free(p);
        for (auto p : acc) tmp_free(p);
        for (auto p : ext_sum) tmp_free(p);
        tmp_free(od_buf);
        tmp_free(od_pt);
        return FHE_OK;
    }

    int act(const MStep &st) {
        fhe_ctx *c = m->ctx;
        const int lv = m->tensors[st.src].level;
        const long long nlN = (long long)(lv + 1) * c->N;
        const int n = B * m->tensors[st.src].n_ct;
        u64 *t3;
        FHE_TRY(tmp(0, (size_t)n * 3 * nlN * 8, &t3));
        FHE_CU(launch_square_act(c->dc, buf[st.src], 2 * nlN, st.c1, st.c0, t3, 3 * nlN, n, lv, s, st.c1v, st.c0v,
                                 m->tensors[st.src].n_ct));
        KsArgs a;
        memset(&a, 0, sizeof(a));
        a.d = t3 + 2 * nlN;
        a.d_item = 3 * nlN;
        a.galois = 1;
        a.key = evk->relin;
        a.key_digits_top = evk->digits;
        a.add0 = t3;
        a.add1 = t3 + nlN;
        a.add_item = 3 * nlN;
        a.out = buf[st.dst];
        a.out_item = 2 * nlN;
        a.n_items = n;
        a.level = lv;
        FHE_TRY(keyswitch(a));
        tmp_free(t3);
        return FHE_OK;
    }

    int rotsum(const MStep &st) {
        const int lv = m->tensors[st.src].level;
        const long long cs = ctst(st.src);
        const int n = B * m->tensors[st.src].n_ct;
        const u64 *cur = buf[st.src];
        u64 *prev_tmp = nullptr;
        if (st.rot.empty()) {
            FHE_CU(cudaMemcpyAsync(buf[st.dst], cur, (size_t)n * cs * 8, cudaMemcpyDeviceToDevice, s));
            return FHE_OK;
        }
        for (size_t k = 0; k < st.rot.size(); k++) {
            u64 *nxt;
            if (k + 1 == st.rot.size()) {
                nxt = buf[st.dst];
            } else {
                FHE_TRY(tmp((int)(k & 1), (size_t)n * cs * 8, &nxt));
            }
            FHE_TRY(rotate_items(cur, cs, st.rot[k], cur, cs, nxt, cs, n, lv));
            if (prev_tmp) tmp_free(prev_tmp);
            prev_tmp = (k + 1 == st.rot.size()) ? nullptr : nxt;
            cur = nxt;
        }
        return FHE_OK;
    }

    int step(int i) {
        const MStep &st = m->steps[i];
        fhe_ctx *c = m->ctx;
        cur_step = i;
        FHE_TRY(alloc_t(st.dst));
        if (st.kind != FHE_STEP_LINEAR) mark(st.kind, true);
        const MTensor &ti = m->tensors[st.src];
        const int n = B * ti.n_ct;
        switch (st.kind) {
        case FHE_STEP_LINEAR:
            FHE_TRY(linear(st));
            break;
        case FHE_STEP_RESCALE:
            FHE_TRY(op_rescale(c, buf[st.src], ctst(st.src), buf[st.dst], ctst(st.dst), n, 2, ti.level, s,
                               pers ? pers->rs_ws : nullptr));
            break;
        case FHE_STEP_ACT:
            FHE_TRY(act(st));
            break;
        case FHE_STEP_ROTSUM:
            FHE_TRY(rotsum(st));
            break;
        case FHE_STEP_CMUL:
            FHE_CU(launch_mul_const(c->dc, buf[st.src], ctst(st.src), st.cval, buf[st.dst], ctst(st.dst), n, 2,
                                    ti.level, s));
            break;
        case FHE_STEP_DROP:
            FHE_CU(launch_drop(c->dc, buf[st.src], ctst(st.src), ti.level, buf[st.dst], ctst(st.dst), st.level, n, 2,
                               s));
            break;
        case FHE_STEP_ADD:
            FHE_CU(launch_add(c->dc, buf[st.src], ctst(st.src), buf[st.src2], ctst(st.src2), buf[st.dst],
                              ctst(st.dst), n, 2, ti.level, 0, s));
            break;
        }
        if (st.kind != FHE_STEP_LINEAR) mark(st.kind, false);
        if (m->last_use[st.src] == i) release(st.src);
        if (st.src2 >= 0 && m->last_use[st.src2] == i) release(st.src2);
        return FHE_OK;
    }
};

int run_steps(Exec &e, int first, int last) {
    for (int i = first; i < last; i++) FHE_TRY(e.step(i));
    return FHE_OK;
}

}  // namespace

static int infer_impl(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, const fhe_ct *const *in, size_t n_img,
                      fhe_ct **out, void *stream, double *ms_by_kind);

extern "C" int fhe_infer(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, const fhe_ct *const *in, size_t n_img,
                         fhe_ct **out, void *stream) {
    return infer_impl(c, mc, evk, in, n_img, out, stream, nullptr);
}

extern "C" int fhe_infer_profiled(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, const fhe_ct *const *in,
                                  size_t n_img, fhe_ct **out, void *stream, double *ms_by_kind) {
    if (!ms_by_kind) return fhe_fail(FHE_E_INVAL, "null argument");
    return infer_impl(c, mc, evk, in, n_img, out, stream, ms_by_kind);
}

static int infer_impl(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, const fhe_ct *const *in, size_t n_img,
                      fhe_ct **out, void *stream, double *ms_by_kind) {
    if (!c || !mc || !evk || !in || !out || n_img == 0) return fhe_fail(FHE_E_INVAL, "null argument");
    fhe_model *m = const_cast<fhe_model *>(mc);
    FHE_CU(cudaSetDevice(c->dev));
    Exec e;
    e.m = m;
    e.evk = evk;
    e.B = (int)n_img;
    e.s = (cudaStream_t)stream;
    e.buf.assign(m->tensors.size(), nullptr);
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
    if (ms_by_kind) e.prof = &prof;
    const MTensor &ti = m->tensors[m->input];
    for (size_t k = 0; k < n_img * ti.n_ct; k++) {
        if (!in[k] || in[k]->level != ti.level || in[k]->n_poly != 2)
            return fhe_fail(FHE_E_LEVEL, "input ciphertext level / shape does not match the model");
    }
    FHE_TRY(e.alloc_t(m->input));
    const long long cs = e.ctst(m->input);
    for (size_t k = 0; k < n_img * ti.n_ct; k++)
        FHE_CU(cudaMemcpyAsync(e.buf[m->input] + k * cs, in[k]->d, cs * 8, cudaMemcpyDeviceToDevice, e.s));
    int rc = run_steps(e, 0, (int)m->steps.size());
    if (rc != FHE_OK) {
        cudaStreamSynchronize(e.s);
        for (auto p : e.buf)
            if (p) cudaFree(p);
        return rc;
    }
    const MTensor &to = m->tensors[m->output];
    const long long cso = e.ctst(m->output);
    std::vector<fhe_ct *> made;
    for (size_t k = 0; k < n_img * to.n_ct; k++) {
        fhe_ct *o = new fhe_ct();
        o->ctx = c;
        o->level = to.level;
        o->n_poly = 2;
        o->scale = to.scale;
        if (dev_alloc(c, (void **)&o->d, cso * 8) != FHE_OK) {
            delete o;
            for (auto p : made) fhe_ct_free(p);
            return FHE_E_OOM;
        }
        cudaMemcpyAsync(o->d, e.buf[m->output] + k * cso, cso * 8, cudaMemcpyDeviceToDevice, e.s);
        made.push_back(o);
    }
    cudaFreeAsync(e.buf[m->output], e.s);
    FHE_CU(cudaStreamSynchronize(e.s));
    if (ms_by_kind) {
        for (int k = 0; k < 16; k++) ms_by_kind[k] = 0;
        for (auto &pr : prof) {
            float ms = 0;
            cudaEventElapsedTime(&ms, pr.second.first, pr.second.second);
            if (pr.first >= 0 && pr.first < 16) ms_by_kind[pr.first] += ms;
            cudaEventDestroy(pr.second.first);
            cudaEventDestroy(pr.second.second);
        }
    }
    for (size_t k = 0; k < made.size(); k++) out[k] = made[k];
    return FHE_OK;
}

// ---- per-step entry points (one image)

static int run_single(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, int step, const fhe_ct *const *in,
                      size_t n_in, fhe_ct **out, size_t n_out, void *stream, int kind_a, int kind_b) {
    if (!c || !mc || !evk || !in || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    fhe_model *m = const_cast<fhe_model *>(mc);
    if (step < 0 || step >= (int)m->steps.size()) return fhe_fail(FHE_E_INVAL, "step index");
    const MStep &st = m->steps[step];
    if (st.kind != kind_a && st.kind != kind_b) return fhe_fail(FHE_E_INVAL, "step has another kind");
    const MTensor &ti = m->tensors[st.src], &to = m->tensors[st.dst];
    if ((int)n_in != ti.n_ct || (int)n_out != to.n_ct) return fhe_fail(FHE_E_INVAL, "ciphertext count");
    for (size_t k = 0; k < n_in; k++)
        if (!in[k] || in[k]->level != ti.level || in[k]->n_poly != 2)
            return fhe_fail(FHE_E_LEVEL, "input level does not match the step");
    FHE_CU(cudaSetDevice(c->dev));
    Exec e;
    e.m = m;
    e.evk = evk;
    e.B = 1;
    e.s = (cudaStream_t)stream;
    e.buf.assign(m->tensors.size(), nullptr);
    FHE_TRY(e.alloc_t(st.src));
    const long long cs = e.ctst(st.src);
    for (size_t k = 0; k < n_in; k++)
        FHE_CU(cudaMemcpyAsync(e.buf[st.src] + k * cs, in[k]->d, cs * 8, cudaMemcpyDeviceToDevice, e.s));
    FHE_TRY(e.alloc_t(st.dst));
    int rc = FHE_OK;
    switch (st.kind) {
    case FHE_STEP_LINEAR: rc = e.linear(st); break;
    case FHE_STEP_ACT: rc = e.act(st); break;
    case FHE_STEP_ROTSUM: rc = e.rotsum(st); break;
    }
    if (rc != FHE_OK) return rc;
    const long long cso = e.ctst(st.dst);
    for (size_t k = 0; k < n_out; k++) {
        fhe_ct *o = new fhe_ct();
        o->ctx = c;
        o->level = to.level;
        o->n_poly = 2;
        o->scale = to.scale;
        FHE_TRY(dev_alloc(c, (void **)&o->d, cso * 8));
        FHE_CU(cudaMemcpyAsync(o->d, e.buf[st.dst] + k * cso, cso * 8, cudaMemcpyDeviceToDevice, e.s));
        out[k] = o;
    }
    FHE_CU(cudaStreamSynchronize(e.s));
    cudaFree(e.buf[st.src]);
    cudaFree(e.buf[st.dst]);
    return FHE_OK;
}

extern "C" int fhe_eval_conv(fhe_ctx *c, const fhe_model *m, const fhe_evk *evk, int step, const fhe_ct *const *in,
                             size_t n_in, fhe_ct **out, size_t n_out, void *stream) {
    return run_single(c, m, evk, step, in, n_in, out, n_out, stream, FHE_STEP_LINEAR, FHE_STEP_LINEAR);
}

extern "C" int fhe_eval_pool_dense(fhe_ctx *c, const fhe_model *m, const fhe_evk *evk, int step,
                                   const fhe_ct *const *in, size_t n_in, fhe_ct **out, size_t n_out, void *stream) {
    return run_single(c, m, evk, step, in, n_in, out, n_out, stream, FHE_STEP_ROTSUM, FHE_STEP_LINEAR);
}

extern "C" int fhe_eval_quad_act(fhe_ctx *c, const fhe_model *m, const fhe_evk *evk, int step, fhe_ct **io, size_t n,
                                 void *stream) {
    std::vector<fhe_ct *> res(n, nullptr);
    FHE_TRY(run_single(c, m, evk, step, (const fhe_ct *const *)io, n, res.data(), n, stream, FHE_STEP_ACT,
                       FHE_STEP_ACT));
    for (size_t k = 0; k < n; k++) {
        std::swap(io[k]->d, res[k]->d);
        io[k]->scale = res[k]->scale;
        fhe_ct_free(res[k]);
    }
    return FHE_OK;
}

// ================================================================ pipeline
//
// Continuous, mixed-level batching.  The program is cut after every
// activation (and the rescale that follows it) into S segments.  Groups of
// `group` images flow through the segments: at each tick every segment k
// processes the group that entered k ticks earlier, so up to S * group images
// at S different levels are in flight, and a new group can enter every tick
// while earlier ones are still on the GPU.  The segments of a tick run
// concurrently on their own streams; each tick's launches are captured once
// per buffer parity into a CUDA graph and replayed.  Tensors live across a cut
// are double-buffered by parity: at tick T segment k reads cut k's buffers
// [T % 2] and writes cut k+1's buffers [(T + 1) % 2].

namespace {

struct Segment {
    int s0 = 0, s1 = 0;
    std::vector<int> ins, outs, pass, internal;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    Persist pers;
    std::map<int, u64 *> ibuf;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // this segment alone, per parity
    long long captured[2] = {0, 0};
};

}  // namespace

struct fhe_pipeline {
    fhe_ctx *ctx = nullptr;
    fhe_model *m = nullptr;
    const fhe_evk *evk = nullptr;
    int g = 1;
    int S = 0;
    bool graphs = true;
    std::vector<int> cuts;
    std::vector<std::map<int, u64 *>> cutbuf[2];
    std::vector<std::unique_ptr<Segment>> seg;
    cudaStream_t main = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long captured[2] = {0, 0};   // kernel launches in each graph
    long long tick = 0;
    std::vector<int> entered;   // images entered at each tick
    std::vector<void *> owned;
    bool creating = false;      // the creation ticks run (and capture) every segment

    ~fhe_pipeline() {
        if (main) cudaStreamSynchronize(main);
        for (auto &e : exec)
            if (e) cudaGraphExecDestroy(e);
        for (auto &sg : seg) {
            for (auto &e : sg->exec)
                if (e) cudaGraphExecDestroy(e);
            if (sg->st) cudaStreamDestroy(sg->st);
            if (sg->done) cudaEventDestroy(sg->done);
        }
        seg.clear();
        if (fork) cudaEventDestroy(fork);
        if (main) cudaStreamDestroy(main);
        for (void *p : owned) cudaFree(p);
    }
};

namespace {

int pipe_alloc(fhe_pipeline *p, size_t bytes, u64 **out) {
    void *d;
    FHE_TRY(dev_alloc(p->ctx, &d, bytes));
    p->owned.push_back(d);
    FHE_CU(cudaMemset(d, 0, bytes));
    *out = (u64 *)d;
    return FHE_OK;
}

int run_segment(fhe_pipeline *p, int k, int parity) {
    Segment &sg = *p->seg[k];
    fhe_model *m = p->m;
    Exec e;
    e.m = m;
    e.evk = p->evk;
    e.B = p->g;
    e.s = sg.st;
    e.buf.assign(m->tensors.size(), nullptr);
    e.pers = &sg.pers;
    sg.pers.variant = parity;
    for (int t : sg.ins) e.buf[t] = p->cutbuf[parity][k].at(t);
    for (int t : sg.outs) e.buf[t] = p->cutbuf[1 - parity][k + 1].at(t);
    for (auto &kv : sg.ibuf) e.buf[kv.first] = kv.second;
    for (int i = sg.s0; i < sg.s1; i++) FHE_TRY(e.step(i));
    for (int t : sg.pass) {
        const size_t bytes = (size_t)p->g * e.item(t) * 8;
        FHE_CU(cudaMemcpyAsync(p->cutbuf[1 - parity][k + 1].at(t), p->cutbuf[parity][k].at(t), bytes,
                               cudaMemcpyDeviceToDevice, sg.st));
    }
    return FHE_OK;
}

// the segments of one tick (occupied[k]: run segment k): fork from the main
// stream, join back into it
int run_tick(fhe_pipeline *p, int parity, const std::vector<char> &occupied) {
    FHE_CU(cudaEventRecord(p->fork, p->main));
    for (int k = 0; k < p->S; k++) {
        if (!occupied[k]) continue;
        FHE_CU(cudaStreamWaitEvent(p->seg[k]->st, p->fork, 0));
        FHE_TRY(run_segment(p, k, parity));
        FHE_CU(cudaEventRecord(p->seg[k]->done, p->seg[k]->st));
    }
    for (int k = 0; k < p->S; k++)
        if (occupied[k]) FHE_CU(cudaStreamWaitEvent(p->main, p->seg[k]->done, 0));
    return FHE_OK;
}

// one segment's launches captured alone on its own stream (per parity)
int capture_segment(fhe_pipeline *p, int k, int parity) {
    Segment &sg = *p->seg[k];
    cudaGraph_t g;
    const unsigned long long l0 = fhe_launch_counter();
    FHE_CU(cudaStreamBeginCapture(sg.st, cudaStreamCaptureModeRelaxed));
    int rc = run_segment(p, k, parity);
    cudaError_t ce = cudaStreamEndCapture(sg.st, &g);
    sg.captured[parity] = (long long)(fhe_launch_counter() - l0);
    fhe_launch_counter_add(-sg.captured[parity]);
    if (rc != FHE_OK) return rc;
    if (ce != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string("segment capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&sg.exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    return FHE_OK;
}

}  // namespace

extern "C" int fhe_pipeline_create(fhe_ctx *c, const fhe_model *mc, const fhe_evk *evk, int group, int use_graphs,
                                   fhe_pipeline **out) {
    if (!c || !mc || !evk || !out || group < 1) return fhe_fail(FHE_E_INVAL, "bad argument");
    fhe_model *m = const_cast<fhe_model *>(mc);
    FHE_CU(cudaSetDevice(c->dev));
    std::unique_ptr<fhe_pipeline> p(new fhe_pipeline());
    p->ctx = c;
    p->m = m;
    p->evk = evk;
    p->g = group;
    p->graphs = use_graphs != 0;
    const int n = (int)m->steps.size();
    // cuts after each activation (after its rescale, when one follows)
    p->cuts.push_back(0);
    for (int i = 0; i < n; i++) {
        if (m->steps[i].kind != FHE_STEP_ACT) continue;
        int c_at = i + 1;
        if (c_at < n && m->steps[c_at].kind == FHE_STEP_RESCALE && m->steps[c_at].src == m->steps[i].dst) c_at++;
        if (c_at < n && c_at > p->cuts.back()) p->cuts.push_back(c_at);
    }
    p->cuts.push_back(n);
    p->S = (int)p->cuts.size() - 1;
    // definition and last use of every tensor
    const int nt = (int)m->tensors.size();
    std::vector<int> def(nt, -2), last(nt, -1);
    def[m->input] = -1;
    for (int i = 0; i < n; i++) {
        def[m->steps[i].dst] = i;
        last[m->steps[i].src] = std::max(last[m->steps[i].src], i);
        if (m->steps[i].src2 >= 0) last[m->steps[i].src2] = std::max(last[m->steps[i].src2], i);
    }
    last[m->output] = n;
    auto live = [&](int cpos) {
        std::vector<int> r;
        for (int t = 0; t < nt; t++)
            if (def[t] >= -1 && def[t] < cpos && last[t] >= cpos) r.push_back(t);
        return r;
    };
    for (int par = 0; par < 2; par++) p->cutbuf[par].resize(p->S + 1);
    for (int ci = 0; ci <= p->S; ci++)
        for (int t : live(p->cuts[ci]))
            for (int par = 0; par < 2; par++) {
                u64 *b;
                FHE_TRY(pipe_alloc(p.get(), (size_t)group * m->tensors[t].n_ct * 2 * (m->tensors[t].level + 1) *
                                                c->N * 8, &b));
                p->cutbuf[par][ci][t] = b;
            }
    FHE_CU(cudaStreamCreateWithFlags(&p->main, cudaStreamNonBlocking));
    FHE_CU(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    for (int k = 0; k < p->S; k++) {
        std::unique_ptr<Segment> sg(new Segment());
        sg->s0 = p->cuts[k];
        sg->s1 = p->cuts[k + 1];
        sg->ins = live(sg->s0);
        std::vector<int> lo = live(sg->s1);
        for (int t : lo) {
            if (def[t] >= sg->s0 && def[t] < sg->s1) sg->outs.push_back(t);
            else sg->pass.push_back(t);
        }
        size_t ks_words = 0, rs_words = 0;
        for (int i = sg->s0; i < sg->s1; i++) {
            const MStep &st = m->steps[i];
            const MTensor &ti = m->tensors[st.src];
            const int t = st.dst;
            if (std::find(lo.begin(), lo.end(), t) == lo.end()) {
                sg->internal.push_back(t);
                u64 *b;
                FHE_TRY(pipe_alloc(p.get(), (size_t)group * m->tensors[t].n_ct * 2 * (m->tensors[t].level + 1) *
                                                c->N * 8, &b));
                sg->ibuf[t] = b;
            }
            int items = 0;
            if (st.kind == FHE_STEP_LINEAR) items = group;
            if (st.kind == FHE_STEP_ACT || st.kind == FHE_STEP_ROTSUM) {
                items = group * ti.n_ct;
                if (c->ks_item_cap > 0) items = std::min(items, c->ks_item_cap);
            }
            ks_words = std::max(ks_words, (size_t)items * ks_workspace_words(c->dc, ti.level));
            if (st.kind == FHE_STEP_RESCALE) rs_words = std::max(rs_words, (size_t)group * ti.n_ct * 2 * (size_t)c->N);
        }
        if (ks_words) FHE_TRY(pipe_alloc(p.get(), ks_words * 8, &sg->pers.ks_ws));
        if (rs_words) FHE_TRY(pipe_alloc(p.get(), rs_words * 8, &sg->pers.rs_ws));
        FHE_CU(cudaStreamCreateWithFlags(&sg->st, cudaStreamNonBlocking));
        FHE_CU(cudaEventCreateWithFlags(&sg->done, cudaEventDisableTiming));
        p->seg.push_back(std::move(sg));
    }
    FHE_CU(cudaDeviceSynchronize());
    if (p->graphs) {
        // capture both parities' graphs now, on an empty pipeline, so that no
        // capture happens later while other threads use the device: the
        // whole tick's, then every segment's alone
        p->creating = true;
        for (int k = 0; k < 4; k++) {
            size_t n_done = 0;
            int64_t tag = -1;
            const int rc = fhe_pipeline_tick(p.get(), nullptr, 0, nullptr, &n_done, &tag);
            if (rc != FHE_OK) return rc;
        }
        p->creating = false;
        for (int par = 0; par < 2; par++)
            for (int k = 0; k < p->S; k++) FHE_TRY(capture_segment(p.get(), k, par));
        FHE_CU(cudaDeviceSynchronize());
        p->tick = 0;
        p->entered.clear();
    }
    *out = p.release();
    return FHE_OK;
}

extern "C" int fhe_pipeline_info(const fhe_pipeline *p, int *n_segments, int *group, int *n_in_ct, int *n_out_ct) {
    if (!p) return fhe_fail(FHE_E_INVAL, "null argument");
    if (n_segments) *n_segments = p->S;
    if (group) *group = p->g;
    if (n_in_ct) *n_in_ct = p->m->tensors[p->m->input].n_ct;
    if (n_out_ct) *n_out_ct = p->m->tensors[p->m->output].n_ct;
    return FHE_OK;
}

// The tick's launches, after its inputs are copied in (see fhe_pipeline_tick).
// Segment k holds the group that entered k ticks ago; segments whose group
// is empty are skipped (a partly filled pipeline, as at low load in
// serving, then costs only its occupied segments).  A full tick replays one
// graph of all segments; a partial one replays the occupied segments' own
// graphs.
static int pipeline_launch(fhe_pipeline *p, int par) {
    std::vector<char> occupied(p->S, 1);
    int n_occ = p->S;
    if (!p->creating) {
        n_occ = 0;
        for (int k = 0; k < p->S; k++) {
            occupied[k] = p->tick - k >= 0 && p->entered[p->tick - k] > 0;
            n_occ += occupied[k];
        }
    }
    if (n_occ == 0) return FHE_OK;
    if (p->graphs && n_occ < p->S && p->seg[0]->exec[par]) {
        FHE_CU(cudaEventRecord(p->fork, p->main));
        for (int k = 0; k < p->S; k++) {
            if (!occupied[k]) continue;
            Segment &sg = *p->seg[k];
            FHE_CU(cudaStreamWaitEvent(sg.st, p->fork, 0));
            FHE_CU(cudaGraphLaunch(sg.exec[par], sg.st));
            fhe_launch_counter_add(sg.captured[par]);
            FHE_CU(cudaEventRecord(sg.done, sg.st));
        }
        for (int k = 0; k < p->S; k++)
            if (occupied[k]) FHE_CU(cudaStreamWaitEvent(p->main, p->seg[k]->done, 0));
        return FHE_OK;
    }
    if (p->graphs && (p->exec[par] || p->tick >= 2)) {
        if (!p->exec[par]) {
            cudaGraph_t g;
            const unsigned long long l0 = fhe_launch_counter();
            FHE_CU(cudaStreamBeginCapture(p->main, cudaStreamCaptureModeRelaxed));
            int rc = run_tick(p, par, occupied);
            cudaError_t ce = cudaStreamEndCapture(p->main, &g);
            p->captured[par] = (long long)(fhe_launch_counter() - l0);
            fhe_launch_counter_add(-p->captured[par]);
            if (rc != FHE_OK) return rc;
            if (ce != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&p->exec[par], g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
        }
        FHE_CU(cudaGraphLaunch(p->exec[par], p->main));
        fhe_launch_counter_add(p->captured[par]);
    } else {
        FHE_TRY(run_tick(p, par, occupied));
    }
    return FHE_OK;
}

// One tick.  Everything that can be refused (arguments, the output
// ciphertexts' memory) is settled before anything is launched, so a refusal
// leaves the pipeline exactly as it was: no group entered, no tick counted,
// and the group due to leave still leaves at the next call.  Once the tick is
// launched it is counted whatever happens next, so the entry ticks of the
// groups inside stay aligned with the tick counter; on a failure after the
// launch *out_tag still names the group that was due to leave (its outputs
// are lost) and *n_out is 0.
extern "C" int fhe_pipeline_tick(fhe_pipeline *p, const fhe_ct *const *in, size_t n_in, fhe_ct **out, size_t *n_out,
                                 int64_t *out_tag) {
    if (!p || !n_out || !out_tag || (n_in && !in) || n_in > (size_t)p->g) return fhe_fail(FHE_E_INVAL, "bad argument");
    *n_out = 0;
    *out_tag = -1;
    fhe_ctx *c = p->ctx;
    fhe_model *m = p->m;
    FHE_CU(cudaSetDevice(c->dev));
    const int par = (int)(p->tick & 1);
    const MTensor &ti = m->tensors[m->input];
    const long long cs_in = 2ll * (ti.level + 1) * c->N;
    for (size_t k = 0; k < n_in * ti.n_ct; k++) {
        if (!in[k] || in[k]->level != ti.level || in[k]->n_poly != 2)
            return fhe_fail(FHE_E_LEVEL, "input ciphertext level / shape does not match the model");
    }
    // the group that entered S-1 ticks ago leaves at this tick: its output
    // ciphertexts are allocated first
    const MTensor &to = m->tensors[m->output];
    const long long cs = 2ll * (to.level + 1) * c->N;
    const long long entry = p->tick - (p->S - 1);
    const int leaving = entry >= 0 ? p->entered[entry] : 0;
    const size_t cnt = (size_t)leaving * to.n_ct;
    for (size_t k = 0; k < cnt; k++) {
        fhe_ct *o = new fhe_ct();
        o->ctx = c;
        o->level = to.level;
        o->n_poly = 2;
        o->scale = to.scale;
        const int rc = dev_alloc(c, (void **)&o->d, cs * 8);
        if (rc != FHE_OK) {
            delete o;
            for (size_t r = 0; r < k; r++) {
                fhe_ct_free(out[r]);
                out[r] = nullptr;
            }
            return rc;
        }
        out[k] = o;
    }
    auto drop_outputs = [&]() {
        for (size_t k = 0; k < cnt; k++) {
            fhe_ct_free(out[k]);
            out[k] = nullptr;
        }
    };
    for (size_t k = 0; k < n_in * ti.n_ct; k++) {
        const cudaError_t e = cudaMemcpyAsync(p->cutbuf[par][0].at(m->input) + k * cs_in, in[k]->d, cs_in * 8,
                                              cudaMemcpyDeviceToDevice, p->main);
        if (e != cudaSuccess) {
            drop_outputs();
            return fhe_fail(FHE_E_CUDA, std::string("input copy: ") + cudaGetErrorString(e));
        }
    }
    p->entered.push_back((int)n_in);
    int rc = pipeline_launch(p, par);
    p->tick++;
    if (leaving > 0) *out_tag = entry;
    if (rc == FHE_OK) {
        const u64 *src = p->cutbuf[1 - par][p->S].at(m->output);
        for (size_t k = 0; k < cnt && rc == FHE_OK; k++) {
            const cudaError_t e = cudaMemcpyAsync(out[k]->d, src + k * cs, cs * 8, cudaMemcpyDeviceToDevice, p->main);
            if (e != cudaSuccess) rc = fhe_fail(FHE_E_CUDA, std::string("output copy: ") + cudaGetErrorString(e));
        }
    }
    const cudaError_t se = cudaStreamSynchronize(p->main);
    if (rc == FHE_OK && se != cudaSuccess) rc = fhe_fail(FHE_E_CUDA, std::string("tick: ") + cudaGetErrorString(se));
    if (rc != FHE_OK) {
        drop_outputs();
        return rc;
    }
    *n_out = (size_t)leaving;
    return FHE_OK;
}

extern "C" int fhe_pipeline_ticks(const fhe_pipeline *p, int64_t *ticks) {
    if (!p || !ticks) return fhe_fail(FHE_E_INVAL, "null argument");
    *ticks = p->tick;
    return FHE_OK;
}

extern "C" int fhe_pipeline_free(fhe_pipeline *p) {
    if (!p) return FHE_OK;
    cudaSetDevice(p->ctx->dev);
    delete p;
    return FHE_OK;
}

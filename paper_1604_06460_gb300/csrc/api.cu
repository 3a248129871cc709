// C ABI (include/qe.h) and the host-side planner: argument checking, the
// gate queue, gate fusion, structure detection and the choice between
// emulating and simulating a subroutine (Sec. III).
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "qe_batch.h"
#include "qe_internal.h"
#include "qe_mlp.h"
#include "qe_plan.h"

namespace {
thread_local std::string g_last_error = "";

int set_error(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}
}  // namespace

#define QE_API_BEGIN try {
#define QE_API_END                                                              \
    return QE_OK;                                                               \
    }                                                                           \
    catch (const qe::Error& e) { return set_error(e.status, e.msg); }           \
    catch (const std::bad_alloc&) { return set_error(QE_ERR_OOM, "host out of memory"); } \
    catch (const std::exception& e) { return set_error(QE_ERR_CUDA, e.what()); } \
    catch (...) { return set_error(QE_ERR_CUDA, "unknown error"); }

namespace qe {

static void check_state(const qe_state* s) {
    if (!s || s->magic != 0x51E57A7E) fail(QE_ERR_STATE, "invalid state handle");
}

static void check_qubits(const qe_state* s, int k, const int* q, uint64_t* mask_out) {
    if (k > 0 && !q) fail(QE_ERR_ARG, "qubit list is NULL");
    uint64_t mask = 0;
    for (int j = 0; j < k; ++j) {
        if (q[j] < 0 || q[j] >= s->n) fail(QE_ERR_ARG, "qubit index out of range");
        if ((mask >> q[j]) & 1ull) fail(QE_ERR_ARG, "duplicate qubit");
        mask |= 1ull << q[j];
    }
    if (mask_out) *mask_out = mask;
}

// ---------------------------------------------------------------- apply
// One block (possibly fused) through the structure-aware dispatch (Sec. II).
void apply_block(qe_state* s, int k, const int* qubits, const std::vector<cd>& U, uint64_t cmask) {
    s->stats.blocks += 1;
    const uint64_t cmask_in = cmask;
    const int D = 1 << k;
    // identity: nothing to do
    bool ident = true;
    for (int r = 0; r < D && ident; ++r)
        for (int c = 0; c < D; ++c)
            if (U[r * D + c] != (r == c ? cd(1.0) : cd(0.0))) { ident = false; break; }
    if (ident) return;
    // strip qubits that act as controls: U is the identity wherever that bit is 0
    std::vector<int> q(qubits, qubits + k);
    std::vector<cd> M = U;
    int kk = k;
    for (int j = kk - 1; j >= 0; --j) {
        const int Dk = 1 << kk;
        bool ctrl = true;
        for (int r = 0; r < Dk && ctrl; ++r)
            for (int c = 0; c < Dk; ++c) {
                if (((r >> j) & 1) && ((c >> j) & 1)) continue;
                cd want = (r == c) ? cd(1.0) : cd(0.0);
                if (M[r * Dk + c] != want) { ctrl = false; break; }
            }
        if (!ctrl) continue;
        // keep the block where bit j = 1
        const int Dn = Dk / 2;
        std::vector<cd> R(Dn * Dn);
        auto ins = [j](int v) { return ((v >> j) << (j + 1)) | (1 << j) | (v & ((1 << j) - 1)); };
        for (int r = 0; r < Dn; ++r)
            for (int c = 0; c < Dn; ++c) R[r * Dn + c] = M[ins(r) * Dk + ins(c)];
        cmask |= 1ull << q[j];
        q.erase(q.begin() + j);
        M.swap(R);
        --kk;
    }
    const int Dk = 1 << kk;
    if (kk == 0) {
        launch_phase_pattern(s, cmask, cmask, M[0]);
        return;
    }
    bool diag = true;
    int nonunit = 0, where = -1;
    for (int r = 0; r < Dk; ++r)
        for (int c = 0; c < Dk; ++c) {
            if (r != c && M[r * Dk + c] != cd(0.0)) diag = false;
            if (r == c && M[r * Dk + c] != cd(1.0)) { ++nonunit; where = r; }
        }
    if (diag && nonunit == 1) {
        uint64_t mask = cmask, value = cmask;
        for (int j = 0; j < kk; ++j) {
            mask |= 1ull << q[j];
            if ((where >> j) & 1) value |= 1ull << q[j];
        }
        launch_phase_pattern(s, mask, value, M[where * Dk + where]);
        return;
    }
    if (diag && cmask == 0) {
        std::vector<cd> d(Dk);
        for (int r = 0; r < Dk; ++r) d[r] = M[r * Dk + r];
        launch_gate_diag(s, kk, q.data(), d.data());
        return;
    }
    // 0/1 permutation matrix: move amplitudes without arithmetic
    bool perm = kk <= 2;
    std::vector<int> p(Dk, -1);
    for (int r = 0; r < Dk && perm; ++r)
        for (int c = 0; c < Dk; ++c) {
            cd v = M[r * Dk + c];
            if (v == cd(1.0)) {
                if (p[r] >= 0) perm = false;
                p[r] = c;
            } else if (v != cd(0.0)) {
                perm = false;
            }
        }
    for (int r = 0; r < Dk && perm; ++r) perm = p[r] >= 0;
    if (perm) {
        launch_permute(s, cmask, kk, q.data(), p.data());
        return;
    }
    if (cmask != 0 && kk <= 2) {
        launch_controlled(s, cmask, kk, q.data(), M.data());
        return;
    }
    if (cmask != 0) {
        // controls found inside a dense block of more than two other qubits:
        // the full matrix already encodes them
        if (cmask_in != 0) fail(QE_ERR_UNSUPPORTED, "controlled gate with more than two targets");
        launch_gate_dense(s, k, qubits, U.data());
        return;
    }
    launch_gate_dense(s, kk, q.data(), M.data());
}

// ----------------------------------------------------------------- fusion
namespace {
}  // namespace

// A fused block ready to run (controls only for gates that came with them).
struct Planned {
    std::vector<int> q;
    std::vector<cd> U;
    uint64_t cmask = 0;
};

// U <- G U, where G acts on the matrix bits pos[0..gk) (row operations on
// the groups of rows that differ only in those bits), in place.
void apply_in_place(std::vector<cd>& U, int D, int gk, const int* pos, const std::vector<cd>& G) {
    const int Dg = 1 << gk;
    int gmask = 0, dep[32];
    for (int j = 0; j < gk; ++j) gmask |= 1 << pos[j];
    for (int c = 0; c < Dg; ++c) {
        int o = 0;
        for (int j = 0; j < gk; ++j)
            if ((c >> j) & 1) o |= 1 << pos[j];
        dep[c] = o;
    }
    // explicit real arithmetic (no library complex multiply); the rows of a
    // group are contiguous runs of D entries
    double* u = reinterpret_cast<double*>(U.data());
    const double* g = reinterpret_cast<const double*>(G.data());
    if (gk == 1) {
        const double g00r = g[0], g00i = g[1], g01r = g[2], g01i = g[3];
        const double g10r = g[4], g10i = g[5], g11r = g[6], g11i = g[7];
        for (int r0 = 0; r0 < D; ++r0) {
            if (r0 & gmask) continue;
            double* a = u + 2 * (size_t)r0 * D;
            double* b = u + 2 * (size_t)(r0 | dep[1]) * D;
            for (int col = 0; col < D; ++col) {
                const double ar = a[2 * col], ai = a[2 * col + 1], br = b[2 * col], bi = b[2 * col + 1];
                a[2 * col] = g00r * ar - g00i * ai + g01r * br - g01i * bi;
                a[2 * col + 1] = g00r * ai + g00i * ar + g01r * bi + g01i * br;
                b[2 * col] = g10r * ar - g10i * ai + g11r * br - g11i * bi;
                b[2 * col + 1] = g10r * ai + g10i * ar + g11r * bi + g11i * br;
            }
        }
        return;
    }
    double xr[32], xi[32];
    for (int r0 = 0; r0 < D; ++r0) {
        if (r0 & gmask) continue;
        for (int col = 0; col < D; ++col) {
            for (int c = 0; c < Dg; ++c) {
                const double* e = u + 2 * ((size_t)(r0 | dep[c]) * D + col);
                xr[c] = e[0];
                xi[c] = e[1];
            }
            for (int r = 0; r < Dg; ++r) {
                double sr = 0.0, si = 0.0;
                const double* gr = g + 2 * (size_t)r * Dg;
                for (int c = 0; c < Dg; ++c) {
                    sr += gr[2 * c] * xr[c] - gr[2 * c + 1] * xi[c];
                    si += gr[2 * c] * xi[c] + gr[2 * c + 1] * xr[c];
                }
                double* e = u + 2 * ((size_t)(r0 | dep[r]) * D + col);
                e[0] = sr;
                e[1] = si;
            }
        }
    }
}

// Frontier fusion: the gates form per-qubit queues; a gate can join a block
// on qubit set S when all its qubits are in S and it is at the front of each
// of their queues (so every gate before it on those qubits is already
// applied or in the block).  Each pass takes the set S (at most max_k qubits)
// that absorbs the most gates: candidate sets are grown from every gate at a
// queue front, adding at each step the qubit, or the remaining qubits of a
// front gate, that lets the block absorb the most gates.  Controlled gates
// and gates wider than max_k stay passes of their own, emitted once they are
// at the front of all their qubits (targets and controls).  Qubits a block
// absorbed no gate on are dropped from it.
void plan_fusion_frontier(const std::vector<PendingGate>& q, int max_k, int nq,
                          const std::function<void(Planned&&)>& emit, bool matrices, bool lookahead) {
    const int G = (int)q.size();
    std::vector<uint64_t> gm(G);      // all qubits of gate i (targets and controls)
    std::vector<char> special(G);
    std::vector<std::vector<int>> queue(nq);
    for (int i = 0; i < G; ++i) {
        uint64_t m = q[i].cmask;
        for (int j = 0; j < q[i].k; ++j) m |= 1ull << q[i].q[j];
        gm[i] = m;
        special[i] = (q[i].cmask != 0 || q[i].k > max_k) ? 1 : 0;
        for (int b = 0; b < nq; ++b)
            if ((m >> b) & 1ull) queue[b].push_back(i);
    }
    std::vector<int> ptr(nq, 0);
    auto front = [&](int b, const std::vector<int>& p) { return p[b] < (int)queue[b].size() ? queue[b][p[b]] : -1; };
    // gates absorbable into a block on S from positions p (p is advanced)
    auto absorb = [&](uint64_t S, std::vector<int>& p, std::vector<int>* taken) {
        int count = 0;
        bool progress = true;
        while (progress) {
            progress = false;
            for (uint64_t r = S; r; r &= r - 1) {
                const int b = __builtin_ctzll(r);
                for (;;) {
                    const int gi = front(b, p);
                    if (gi < 0 || special[gi] || (gm[gi] & ~S)) break;
                    bool at_front = true;
                    for (uint64_t t = gm[gi]; t; t &= t - 1)
                        if (front(__builtin_ctzll(t), p) != gi) { at_front = false; break; }
                    if (!at_front) break;
                    for (uint64_t t = gm[gi]; t; t &= t - 1) ++p[__builtin_ctzll(t)];
                    if (taken) taken->push_back(gi);
                    ++count;
                    progress = true;
                }
            }
        }
        return count;
    };
    // Absorption is confluent (taking a gate never blocks another), so the
    // gates of S | add are those of S plus what absorbing S | add from S's
    // end positions adds.
    std::vector<int> pS(nq), scratch(nq);
    // grow a candidate set from S up to max_k qubits with the queues at
    // positions base; returns its gate count
    auto grow = [&](uint64_t& S, const std::vector<int>& base) {
        pS = base;
        int cS = absorb(S, pS, nullptr);
        while (__builtin_popcountll(S) < max_k) {
            int best = -1, best_add = 0;
            uint64_t best_m = 0;
            auto consider = [&](uint64_t add) {
                if (!add || __builtin_popcountll(S | add) > max_k) return;
                scratch = pS;
                const int sc = cS + absorb(S | add, scratch, nullptr), na = __builtin_popcountll(add);
                if (sc > best || (sc == best && na < best_add)) { best = sc; best_add = na; best_m = add; }
            };
            for (int b = 0; b < nq; ++b) {
                if (((S >> b) & 1ull) || base[b] >= (int)queue[b].size()) continue;
                consider(1ull << b);
                const int gi = queue[b][base[b]];
                if (!special[gi]) consider(gm[gi] & ~S);
            }
            if (best < 0) break;
            S |= best_m;
            cS += absorb(S, pS, nullptr);
        }
        return cS;
    };
    // (gate count, set) of the set grown from each distinct front gate
    auto candidates = [&](const std::vector<int>& base, std::vector<std::pair<int, uint64_t>>& out) {
        out.clear();
        for (int b = 0; b < nq; ++b) {
            const int gi = front(b, base);
            if (gi < 0 || special[gi]) continue;
            uint64_t S = gm[gi];
            bool dup = false;   // the same front gate seen from another of its qubits
            for (int c = 0; c < b && !dup; ++c) {
                const int gc = front(c, base);
                dup = gc >= 0 && !special[gc] && gm[gc] == gm[gi];
            }
            if (dup) continue;
            const int cnt = grow(S, base);
            out.emplace_back(cnt, S);
        }
    };
    std::vector<std::pair<int, uint64_t>> cand, next;
    std::vector<int> after(nq);
    int remaining = G;
    std::vector<int> taken;
    while (remaining > 0) {
        // standalone gates that are ready go first
        bool emitted = false;
        for (int b = 0; b < nq && !emitted; ++b) {
            const int gi = front(b, ptr);
            if (gi < 0 || !special[gi]) continue;
            bool ready = true;
            for (uint64_t t = gm[gi]; t; t &= t - 1)
                if (front(__builtin_ctzll(t), ptr) != gi) { ready = false; break; }
            if (!ready) continue;
            Planned p;
            p.q.assign(q[gi].q, q[gi].q + q[gi].k);
            if (matrices) p.U = q[gi].U;
            p.cmask = q[gi].cmask;
            for (uint64_t t = gm[gi]; t; t &= t - 1) ++ptr[__builtin_ctzll(t)];
            --remaining;
            emitted = true;
            emit(std::move(p));
        }
        if (emitted) continue;
        // the best block over the sets grown from each front gate; with
        // look-ahead, the sets are ranked by their own gate count plus that
        // of the best block after them
        candidates(ptr, cand);
        uint64_t bestS = 0;
        int bestc = -1;
        for (auto& [c, S] : cand)
            if (c > bestc || (c == bestc && __builtin_popcountll(S) < __builtin_popcountll(bestS))) {
                bestc = c;
                bestS = S;
            }
        if (lookahead && cand.size() > 1) {
            std::sort(cand.begin(), cand.end(), [](const std::pair<int, uint64_t>& x, const std::pair<int, uint64_t>& y) {
                return x.first != y.first ? x.first > y.first
                                          : __builtin_popcountll(x.second) < __builtin_popcountll(y.second);
            });
            int best_total = -1;
            for (auto& [c, S] : cand) {
                after = ptr;
                absorb(S, after, nullptr);
                candidates(after, next);
                int nb = 0;
                for (auto& x : next) nb = std::max(nb, x.first);
                if (c + nb > best_total) {
                    best_total = c + nb;
                    bestc = c;
                    bestS = S;
                }
            }
        }
        if (bestc <= 0) fail(QE_ERR_STATE, "fusion planner made no progress");
        taken.clear();
        absorb(bestS, ptr, &taken);
        uint64_t used = 0;
        for (int gi : taken) used |= gm[gi];
        Planned p;
        for (uint64_t t = used; t; t &= t - 1) p.q.push_back(__builtin_ctzll(t));
        if (matrices) {
            const int D = 1 << p.q.size();
            p.U.assign((size_t)D * D, 0.0);
            for (int r = 0; r < D; ++r) p.U[(size_t)r * D + r] = 1.0;
            for (int gi : taken) {
                int pos[5];
                for (int j = 0; j < q[gi].k; ++j)
                    pos[j] = (int)(std::find(p.q.begin(), p.q.end(), q[gi].q[j]) - p.q.begin());
                apply_in_place(p.U, D, q[gi].k, pos, q[gi].U);
            }
        }
        remaining -= (int)taken.size();
        emit(std::move(p));
    }
}

// The fused passes for the queued gates, handed to `emit` in order as they
// are planned (so the caller can launch each while the next is planned).
// max_k <= 1: no fusion, every gate is its own pass.  Without `matrices` only
// the qubit sets are produced.
void plan_fusion(const std::vector<PendingGate>& q, int max_k, int nq, const std::function<void(Planned&&)>& emit,
                 bool matrices = true, bool lookahead = false) {
    if (max_k <= 1) {
        for (auto& g : q) {
            Planned p;
            p.q.assign(g.q, g.q + g.k);
            if (matrices) p.U = g.U;
            p.cmask = g.cmask;
            emit(std::move(p));
        }
        return;
    }
    plan_fusion_frontier(q, max_k, nq, emit, matrices, lookahead);
}

std::vector<Planned> plan_fusion_list(const std::vector<PendingGate>& q, int max_k, int nq, bool matrices,
                                      bool lookahead) {
    std::vector<Planned> out;
    plan_fusion(q, max_k, nq, [&](Planned&& p) { out.push_back(std::move(p)); }, matrices, lookahead);
    return out;
}

// Look-ahead costs about ten times the planning (~3 ms per block for 900
// gates on 30 qubits, against ~0.3 ms); it is used from 2^30 amplitudes on,
// where a pass is long enough for the planning of the next block to hide
// behind it.  On seven random circuits of 28-32 qubits it takes 2 % fewer
// blocks in all (never more on any of them).
bool plan_lookahead(int n) { return n >= 30; }

uint32_t* status_word_host(qe_state* s) {
    if (!s->status_host) {
        QE_CUDA(cudaMallocHost(&s->status_host, sizeof(uint32_t)));
        *s->status_host = 0u;
    }
    return s->status_host;
}

void complete_pending(qe_state* s) {
    if (!s->status_pending) return;
    s->status_pending = false;
    QE_CUDA(cudaStreamSynchronize(s->stream));
    const uint32_t st = *s->status_host;
    *s->status_host = 0u;
    if (st) fail(QE_ERR_TIMEOUT, "tensor-core gate: an mbarrier wait exceeded its limit");
}


void flush(qe_state* s) {
    if (s->queue.empty()) {
        complete_pending(s);   // a tensor-core pass launched outside a flush (QFT digit passes)
        return;
    }
    std::vector<PendingGate> q;
    q.swap(s->queue);
    const int k = choose_fusion_width(s, q);
    s->stats.gates += q.size();
    try {
        plan_fusion(
            q, k, s->n, [&](Planned&& b) { apply_block(s, (int)b.q.size(), b.q.data(), b.U, b.cmask); }, true,
            plan_lookahead(s->n));
    } catch (...) {
        try {
            complete_pending(s);
        } catch (...) {
        }
        throw;
    }
    complete_pending(s);
}

// Fusion width: the state's max_k, or, under QE_POLICY_AUTO with a learned
// model, the width in [1, max_k] whose planned blocks the model predicts to
// run fastest (sum over blocks of the predicted pass time).
int choose_fusion_width(qe_state* s, const std::vector<PendingGate>& q) {
    if (s->policy != QE_POLICY_AUTO || !s->model || q.empty() || s->max_k <= 1) return s->max_k;
    std::vector<float> X;
    std::vector<int> owner;
    for (int k = 1; k <= s->max_k; ++k) {
        for (auto& b : plan_fusion_list(q, k, s->n, false, false)) {
            int lo = s->n, hi = 0;
            for (int v : b.q) { lo = std::min(lo, v); hi = std::max(hi, v); }
            for (int j = 0; j < s->n; ++j)
                if ((b.cmask >> j) & 1ull) { lo = std::min(lo, j); hi = std::max(hi, j); }
            float f[kCostFeatures];
            cost_features(kOpGatePass, s->n, s->dtype, (int)b.q.size(), lo, hi, 0, 0, f);
            X.insert(X.end(), f, f + kCostFeatures);
            owner.push_back(k);
        }
    }
    std::vector<float> y(owner.size());
    mlp_predict(s->model, X.data(), (int)owner.size(), y.data());
    std::vector<double> total(s->max_k + 1, 0.0);
    for (size_t i = 0; i < owner.size(); ++i) total[owner[i]] += std::exp((double)y[i]);
    int best = 1;
    for (int k = 2; k <= s->max_k; ++k)
        if (total[k] < total[best]) best = k;
    return best;
}

// ------------------------------------------------------------ subroutines
static void qft_simulated(qe_state* s, int lo, int m, int inverse) {
    const double r2 = 1.0 / std::sqrt(2.0);
    std::vector<cd> H = {r2, r2, r2, -r2};
    // CR(theta) = diag(1, 1, 1, e^{i theta}) on (target, control) (Table I)
    auto cr = [&](int c, int t, double th) {
        std::vector<cd> D(16, 0.0);
        D[0] = 1.0;
        D[5] = 1.0;
        D[10] = 1.0;
        D[15] = std::polar(1.0, th);
        int qq[2] = {t, c};
        apply_block(s, 2, qq, D, 0);
    };
    if (!inverse) {
        for (int j = m - 1; j >= 0; --j) {
            int qj = lo + j;
            apply_block(s, 1, &qj, H, 0);
            for (int l = j - 1; l >= 0; --l) cr(lo + l, lo + j, M_PI / std::ldexp(1.0, j - l));
        }
        launch_bitrev(s, lo, m);
    } else {
        launch_bitrev(s, lo, m);
        for (int j = 0; j < m; ++j) {
            for (int l = 0; l < j; ++l) cr(lo + l, lo + j, -M_PI / std::ldexp(1.0, j - l));
            int qj = lo + j;
            apply_block(s, 1, &qj, H, 0);
        }
    }
    s->stats.gates += (uint64_t)m + (uint64_t)m * (m - 1) / 2;
}

// c += a b as multi-controlled NOTs (repeated addition and shift, Sec. III-A):
// for every pair of bits a_i, b_j with i + j < N, an increment of the
// sub-register c[i+j ..] under the controls a_i, b_j.
static void mul_simulated(qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; i + j < N; ++j)
            for (int k = N - 1; k >= i + j; --k) {
                uint64_t cm = (1ull << qa[i]) | (1ull << qb[j]);
                for (int l = i + j; l < k; ++l) cm |= 1ull << qc[l];
                int t = qc[k];
                int perm[2] = {1, 0};
                launch_permute(s, cm, 1, &t, perm);
                s->stats.gates += 1;
            }
}

static void add_simulated(qe_state* s, int m, const int* qubits, uint64_t c) {
    // ripple of multi-controlled NOTs: adding 2^j increments (qubits[j..m-1])
    for (int j = 0; j < m; ++j) {
        if (!((c >> j) & 1ull)) continue;
        for (int i = m - 1; i >= j; --i) {
            uint64_t cm = 0;
            for (int l = j; l < i; ++l) cm |= 1ull << qubits[l];
            int t = qubits[i];
            int perm[2] = {1, 0};
            launch_permute(s, cm, 1, &t, perm);
            s->stats.gates += 1;
        }
    }
}

}  // namespace qe

// =================================================================== C ABI
using namespace qe;

static void check_batch(const qe_batch* b) {
    if (!b || b->magic != 0xBA7C4) fail(QE_ERR_STATE, "invalid batch handle");
}

extern "C" {

int qe_plan_fusion(int n, int ngates, const int* k, const int* qubits, const double* matrices,
                   const int64_t* mat_offset, int max_k, int cap, int* nblocks, int* block_k,
                   int* block_qubits, double* block_matrices) {
    QE_API_BEGIN
    if (n < 1 || n > 34) fail(QE_ERR_ARG, "n must be in [1, 34]");
    if (ngates < 0 || (ngates > 0 && (!k || !qubits || !matrices || !mat_offset)))
        fail(QE_ERR_ARG, "gate arrays are NULL");
    if (max_k < 1 || max_k > 5) fail(QE_ERR_ARG, "max_k must be in [1, 5]");
    if (!nblocks) fail(QE_ERR_ARG, "nblocks is NULL");
    std::vector<PendingGate> q(ngates);
    for (int g = 0; g < ngates; ++g) {
        if (k[g] < 1 || k[g] > 5) fail(QE_ERR_ARG, "gate width must be in [1, 5]");
        q[g].k = k[g];
        uint64_t seen = 0;
        for (int j = 0; j < k[g]; ++j) {
            const int qq = qubits[5 * g + j];
            if (qq < 0 || qq >= n || ((seen >> qq) & 1ull)) fail(QE_ERR_ARG, "qubit out of range or repeated");
            seen |= 1ull << qq;
            q[g].q[j] = qq;
        }
        const int D = 1 << k[g];
        q[g].U.resize((size_t)D * D);
        const double* m = matrices + mat_offset[g];
        for (int i = 0; i < D * D; ++i) q[g].U[i] = cd(m[2 * i], m[2 * i + 1]);
    }
    const std::vector<Planned> plan = plan_fusion_list(q, max_k, n, true, plan_lookahead(n));
    *nblocks = (int)plan.size();
    if ((int)plan.size() > cap) fail(QE_ERR_ARG, "more blocks than cap");
    if (!plan.empty() && (!block_k || !block_qubits || !block_matrices)) fail(QE_ERR_ARG, "output arrays are NULL");
    for (size_t b = 0; b < plan.size(); ++b) {
        const int kb = (int)plan[b].q.size();
        block_k[b] = kb;
        for (int j = 0; j < 5; ++j) block_qubits[5 * b + j] = j < kb ? plan[b].q[j] : -1;
        for (size_t i = 0; i < plan[b].U.size(); ++i) {
            block_matrices[2048 * b + 2 * i] = plan[b].U[i].real();
            block_matrices[2048 * b + 2 * i + 1] = plan[b].U[i].imag();
        }
    }
    QE_API_END
}

const char* qe_last_error(void) { return g_last_error.c_str(); }

// Default fusion width: 5-qubit blocks where the tensor cores take them
// (n >= 12, not the native-FP64 baseline), else 2 (complex128) / 4 (complex64).
static int default_fusion_width(const qe_state* s) {
    const bool tc_blocks = s->tensor_cores && !s->force_tile && s->n >= 12 &&
                           !(s->dtype == QE_C128 && !s->c128_tc);
    return tc_blocks ? 5 : (s->dtype == QE_C128 ? 2 : 4);
}

int qe_alloc_state(int n, int dtype, void* dev_ptr, size_t bytes, void* stream, qe_state** out) {
    QE_API_BEGIN
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 34) fail(QE_ERR_ARG, "n must be in [1, 34]");
    if (dtype != QE_C64 && dtype != QE_C128) fail(QE_ERR_ARG, "unknown dtype");
    const size_t need = (size_t)(dtype == QE_C128 ? 16 : 8) << n;
    auto* s = new qe_state();
    s->n = n;
    s->dtype = dtype;
    s->stream = (cudaStream_t)stream;
    // QE_C128_ARITH: "df64" selects the double-float mode, "f64" the FP64
    // mode without tensor cores (the native-FP64 baseline); unset: FP64 mode
    const char* ar = std::getenv("QE_C128_ARITH");
    s->arith = (ar && std::strcmp(ar, "df64") == 0) ? QE_ARITH_DF64 : QE_ARITH_FP64;
    s->c128_tc = (ar && std::strcmp(ar, "f64") == 0) ? 0 : 1;
    const char* tl = std::getenv("QE_DENSE_TILE");
    s->force_tile = (tl && std::strcmp(tl, "1") == 0) ? 1 : 0;
    const char* tc = std::getenv("QE_TENSOR_CORES");
    s->tensor_cores = (tc && std::strcmp(tc, "0") == 0) ? 0 : 1;
    s->max_k = default_fusion_width(s);
    try {
        if (dev_ptr) {
            if (bytes < need) fail(QE_ERR_ARG, "borrowed buffer too small");
            if (((uintptr_t)dev_ptr) & 255u) fail(QE_ERR_ARG, "borrowed buffer not 256-byte aligned");
            s->d = dev_ptr;
            s->owned = false;
        } else {
            cudaError_t e = cudaMalloc(&s->d, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                fail(QE_ERR_OOM, std::string("cudaMalloc of the state failed: ") + cudaGetErrorString(e));
            }
            s->owned = true;
        }
        s->bytes = need;
        launch_init_basis(s, 0);
        QE_CUDA(cudaStreamSynchronize(s->stream));
    } catch (...) {
        if (s->owned && s->d) cudaFree(s->d);
        delete s;
        throw;
    }
    *out = s;
    QE_API_END
}

int qe_free_state(qe_state* s) {
    QE_API_BEGIN
    if (!s) return QE_OK;
    check_state(s);
    cudaStreamSynchronize(s->stream);
    if (s->owned && s->d) cudaFree(s->d);
    if (s->scratch) cudaFree(s->scratch);
    if (s->oz_ws) cudaFree(s->oz_ws);
    if (s->status_host) cudaFreeHost(s->status_host);
    profile_clear(s);
    for (auto e : s->event_pool) cudaEventDestroy(e);
    s->magic = 0;
    delete s;
    QE_API_END
}

int qe_state_info(const qe_state* s, int* n, int* dtype, void** dev_ptr) {
    QE_API_BEGIN
    check_state(s);
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    if (dev_ptr) *dev_ptr = s->d;
    QE_API_END
}

int qe_init_basis(qe_state* s, uint64_t index) {
    QE_API_BEGIN
    check_state(s);
    if (index >= dim(s)) fail(QE_ERR_ARG, "basis index out of range");
    s->queue.clear();
    launch_init_basis(s, index);
    QE_API_END
}

int qe_init_random(qe_state* s, uint64_t seed) {
    QE_API_BEGIN
    check_state(s);
    s->queue.clear();
    launch_init_random(s, seed);
    QE_API_END
}

int qe_set_amplitudes(qe_state* s, const void* host, uint64_t offset, uint64_t count) {
    QE_API_BEGIN
    check_state(s);
    if (!host && count) fail(QE_ERR_ARG, "host is NULL");
    if (offset > dim(s) || count > dim(s) - offset) fail(QE_ERR_ARG, "range out of bounds");
    flush(s);
    QE_CUDA(cudaMemcpyAsync((char*)s->d + offset * amp_bytes(s), host, count * amp_bytes(s),
                            cudaMemcpyHostToDevice, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    QE_API_END
}

int qe_get_amplitudes(qe_state* s, void* host, uint64_t offset, uint64_t count) {
    QE_API_BEGIN
    check_state(s);
    if (!host && count) fail(QE_ERR_ARG, "host is NULL");
    if (offset > dim(s) || count > dim(s) - offset) fail(QE_ERR_ARG, "range out of bounds");
    flush(s);
    QE_CUDA(cudaMemcpyAsync(host, (const char*)s->d + offset * amp_bytes(s), count * amp_bytes(s),
                            cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    QE_API_END
}

int qe_apply_gate(qe_state* s, int k, const int* qubits, const double* matrix) {
    QE_API_BEGIN
    check_state(s);
    if (k < 1 || k > 5) fail(QE_ERR_ARG, "k must be in [1, 5]");
    check_qubits(s, k, qubits, nullptr);
    if (!matrix) fail(QE_ERR_ARG, "matrix is NULL");
    PendingGate g;
    g.k = k;
    for (int j = 0; j < k; ++j) g.q[j] = qubits[j];
    const int D = 1 << k;
    g.U.resize(D * D);
    for (int i = 0; i < D * D; ++i) {
        if (!std::isfinite(matrix[2 * i]) || !std::isfinite(matrix[2 * i + 1]))
            fail(QE_ERR_ARG, "matrix has a non-finite entry");
        g.U[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
    }
    s->queue.push_back(std::move(g));
    QE_API_END
}

int qe_apply_controlled(qe_state* s, int nc, const int* controls, int k, const int* targets,
                        const double* matrix) {
    QE_API_BEGIN
    check_state(s);
    if (nc < 0 || k < 0 || k > 2) fail(QE_ERR_ARG, "need nc >= 0 and 0 <= k <= 2");
    uint64_t cm = 0, tm = 0;
    check_qubits(s, nc, controls, &cm);
    check_qubits(s, k, targets, &tm);
    if (cm & tm) fail(QE_ERR_ARG, "a qubit is both control and target");
    if (!matrix) fail(QE_ERR_ARG, "matrix is NULL");
    PendingGate g;
    g.k = k;
    for (int j = 0; j < k; ++j) g.q[j] = targets[j];
    g.cmask = cm;
    const int D = 1 << k;
    g.U.resize(D * D);
    for (int i = 0; i < D * D; ++i) g.U[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
    if (k == 0 && cm == 0) fail(QE_ERR_ARG, "a global phase needs at least one control");
    if (k == 0) {
        flush(s);
        launch_phase_pattern(s, cm, cm, g.U[0]);
        s->stats.gates += 1;
    } else {
        s->queue.push_back(std::move(g));
    }
    QE_API_END
}

int qe_apply_qft(qe_state* s, int lo, int m, int inverse) {
    QE_API_BEGIN
    check_state(s);
    if (m < 1 || lo < 0 || lo + m > s->n) fail(QE_ERR_ARG, "register [lo, lo+m) out of range");
    flush(s);
    if (choose_emulate_qft(s, lo, m)) launch_qft_fft(s, lo, m, inverse);
    else qft_simulated(s, lo, m, inverse);
    QE_API_END
}

int qe_apply_add_const(qe_state* s, int m, const int* qubits, uint64_t c) {
    QE_API_BEGIN
    check_state(s);
    if (m < 1 || m > s->n) fail(QE_ERR_ARG, "m out of range");
    check_qubits(s, m, qubits, nullptr);
    flush(s);
    if (choose_emulate_add(s, m, qubits, c)) launch_add_const(s, m, qubits, c);
    else add_simulated(s, m, qubits, c);
    QE_API_END
}

static void check_arith_registers(const qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    if (N < 1 || N > 16 || 3 * N > s->n) fail(QE_ERR_ARG, "register width N must be in [1, min(16, n/3)]");
    uint64_t ma = 0, mb = 0, mc = 0;
    check_qubits(s, N, qa, &ma);
    check_qubits(s, N, qb, &mb);
    check_qubits(s, N, qc, &mc);
    if ((ma & mb) || (ma & mc) || (mb & mc)) fail(QE_ERR_ARG, "registers a, b, c overlap");
}

int qe_apply_mul(qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    QE_API_BEGIN
    check_state(s);
    check_arith_registers(s, N, qa, qb, qc);
    flush(s);
    if (choose_emulate_mul(s, N)) launch_mul(s, N, qa, qb, qc);
    else mul_simulated(s, N, qa, qb, qc);
    QE_API_END
}

int qe_apply_div(qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    QE_API_BEGIN
    check_state(s);
    check_arith_registers(s, N, qa, qb, qc);
    if (s->policy == QE_POLICY_SIMULATE)
        fail(QE_ERR_UNSUPPORTED, "the division is only emulated (its reversible circuit needs work qubits)");
    flush(s);
    launch_div(s, N, qa, qb, qc);
    QE_API_END
}

int qe_expectation(qe_state* s, int nterms, const uint64_t* xmask, const uint64_t* zmask,
                   const double* coeff, double* out) {
    QE_API_BEGIN
    check_state(s);
    if (nterms < 0 || (nterms && (!xmask || !zmask || !coeff)) || !out) fail(QE_ERR_ARG, "bad term arrays");
    const uint64_t valid = (s->n >= 64) ? ~0ull : ((1ull << s->n) - 1ull);
    for (int t = 0; t < nterms; ++t) {
        if ((xmask[t] | zmask[t]) & ~valid) fail(QE_ERR_ARG, "Pauli mask names a qubit >= n");
        if (!std::isfinite(coeff[t])) fail(QE_ERR_ARG, "non-finite coefficient");
    }
    flush(s);
    *out = reduce_expectation(s, nterms, xmask, zmask, coeff);
    QE_API_END
}

int qe_probs(qe_state* s, int m, const int* qubits, double* out) {
    QE_API_BEGIN
    check_state(s);
    if (m < 1 || m > 16 || m > s->n) fail(QE_ERR_ARG, "m must be in [1, min(16, n)]");
    check_qubits(s, m, qubits, nullptr);
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    flush(s);
    reduce_probs(s, m, qubits, out);
    QE_API_END
}

int qe_init_identity(qe_state* s, int nsys) {
    QE_API_BEGIN
    check_state(s);
    if (s->dtype != QE_C128) fail(QE_ERR_ARG, "dense matrices are complex128 states");
    if (nsys < 1 || 2 * nsys != s->n) fail(QE_ERR_ARG, "the state must have 2 nsys qubits");
    s->queue.clear();
    launch_init_identity(s, nsys);
    QE_API_END
}

static void check_matrix_state(const qe_state* m, int k) {
    check_state(m);
    if (m->dtype != QE_C128 || m->n != 2 * k) fail(QE_ERR_ARG, "matrix states must be complex128 of 2k qubits");
}

int qe_matmul(qe_state* c, qe_state* a, qe_state* b) {
    QE_API_BEGIN
    check_state(c);
    const int k = c->n / 2;
    if (c->n % 2 || k < 1) fail(QE_ERR_ARG, "matrix states must have an even number of qubits");
    check_matrix_state(a, k);
    check_matrix_state(b, k);
    if (c == a || c == b || c->d == a->d || c->d == b->d) fail(QE_ERR_ARG, "the product may not overwrite a factor");
    flush(a);
    flush(b);
    flush(c);
    if (a->stream != c->stream) QE_CUDA(cudaStreamSynchronize(a->stream));
    if (b->stream != c->stream && b->stream != a->stream) QE_CUDA(cudaStreamSynchronize(b->stream));
    launch_matmul(c, c->d, a->d, b->d, k);
    QE_API_END
}

int qe_qpe_emulate(qe_state* s, int nsys, int b, qe_state* u) {
    QE_API_BEGIN
    check_state(s);
    check_matrix_state(u, nsys);
    if (s->dtype != QE_C128) fail(QE_ERR_ARG, "phase estimation runs on complex128 states");
    if (b < 1 || nsys < 1 || nsys + b > s->n) fail(QE_ERR_ARG, "need 1 <= b and nsys + b <= n");
    if (u == s || u->d == s->d) fail(QE_ERR_ARG, "the matrix state may not be the state");
    flush(u);
    flush(s);
    if (u->stream != s->stream) QE_CUDA(cudaStreamSynchronize(u->stream));
    // Hadamards on the ancillas [nsys, nsys + b)
    const double r2 = 1.0 / std::sqrt(2.0);
    const std::vector<cd> H = {r2, r2, r2, -r2};
    for (int j = 0; j < b; ++j) {
        const int q = nsys + j;
        apply_block(s, 1, &q, H, 0);
    }
    // ancilla j controls U^(2^j): the powers by repeated squaring in two
    // temporary matrices
    const size_t mbytes = (size_t)16 << (2 * nsys);
    void* tmp[2] = {nullptr, nullptr};
    if (b > 1) {
        for (auto& t : tmp) {
            cudaError_t e = cudaMalloc(&t, mbytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (tmp[0]) cudaFree(tmp[0]);
                fail(QE_ERR_OOM, "no room for the matrix powers");
            }
        }
    }
    try {
        const void* cur = u->d;
        for (int j = 0; j < b; ++j) {
            launch_dense_controlled(s, cur, nsys, nsys + j);
            if (j + 1 < b) {
                void* next = tmp[j & 1];
                launch_matmul(s, next, cur, cur, nsys);
                cur = next;
            }
        }
        launch_qft_fft(s, nsys, b, 1);
        QE_CUDA(cudaStreamSynchronize(s->stream));
    } catch (...) {
        cudaStreamSynchronize(s->stream);
        for (auto t : tmp)
            if (t) cudaFree(t);
        throw;
    }
    for (auto t : tmp)
        if (t) cudaFree(t);
    QE_API_END
}

int qe_sample(qe_state* s, int m, const int* qubits, int nshots, const double* uniforms, uint64_t* outcomes) {
    QE_API_BEGIN
    check_state(s);
    if (m < 0 || m > 16 || m > s->n) fail(QE_ERR_ARG, "m must be 0 (all qubits) or in [1, min(16, n)]");
    if (m > 0) check_qubits(s, m, qubits, nullptr);
    if (nshots < 0 || (nshots > 0 && (!uniforms || !outcomes))) fail(QE_ERR_ARG, "bad shot arrays");
    for (int i = 0; i < nshots; ++i)
        if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) fail(QE_ERR_ARG, "uniforms must lie in [0, 1)");
    flush(s);
    sample_shots(s, m, qubits, nshots, uniforms, outcomes);
    QE_API_END
}

int qe_collapse(qe_state* s, int m, const int* qubits, uint64_t outcome, double* probability) {
    QE_API_BEGIN
    check_state(s);
    if (m < 1 || m > s->n) fail(QE_ERR_ARG, "m must be in [1, n]");
    check_qubits(s, m, qubits, nullptr);
    if (m < 64 && (outcome >> m) != 0) fail(QE_ERR_ARG, "outcome has bits beyond the m measured qubits");
    flush(s);
    const double p = collapse(s, m, qubits, outcome);
    if (probability) *probability = p;
    QE_API_END
}

int qe_norm2(qe_state* s, double* out) {
    QE_API_BEGIN
    check_state(s);
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    flush(s);
    *out = reduce_norm2(s);
    QE_API_END
}

int qe_flush(qe_state* s) {
    QE_API_BEGIN
    check_state(s);
    flush(s);
    QE_API_END
}

int qe_sync(qe_state* s) {
    QE_API_BEGIN
    check_state(s);
    flush(s);
    QE_CUDA(cudaStreamSynchronize(s->stream));
    QE_API_END
}

int qe_set_policy(qe_state* s, int policy, int max_k) {
    QE_API_BEGIN
    check_state(s);
    if (policy < QE_POLICY_AUTO || policy > QE_POLICY_SIMULATE) fail(QE_ERR_ARG, "unknown policy");
    if (max_k < 0 || max_k > 5) fail(QE_ERR_ARG, "max_k must be in [0, 5]");
    flush(s);
    s->policy = policy;
    s->max_k = max_k == 0 ? default_fusion_width(s) : max_k;
    QE_API_END
}

int qe_set_arith(qe_state* s, int arith) {
    QE_API_BEGIN
    check_state(s);
    if (arith != QE_ARITH_FP64 && arith != QE_ARITH_DF64) fail(QE_ERR_ARG, "unknown arithmetic mode");
    flush(s);
    QE_CUDA(cudaStreamSynchronize(s->stream));
    const bool keep_k = s->max_k != default_fusion_width(s);
    s->arith = arith;
    if (!keep_k) s->max_k = default_fusion_width(s);
    QE_API_END
}

int qe_get_arith(const qe_state* s, int* arith) {
    QE_API_BEGIN
    check_state(s);
    if (!arith) fail(QE_ERR_ARG, "arith is NULL");
    *arith = s->arith;
    QE_API_END
}

int qe_get_stats(const qe_state* s, qe_stats* out) {
    QE_API_BEGIN
    check_state(s);
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    out->launches = s->stats.launches;
    out->passes = s->stats.passes;
    out->algorithmic_bytes = s->stats.bytes;
    out->gates_applied = s->stats.gates;
    out->fused_blocks = s->stats.blocks;
    QE_API_END
}

int qe_profile_enable(qe_state* s, int enable) {
    QE_API_BEGIN
    check_state(s);
    flush(s);
    QE_CUDA(cudaStreamSynchronize(s->stream));
    profile_clear(s);
    s->profile = enable != 0;
    QE_API_END
}

int qe_profile_read(qe_state* s, qe_kernel_profile* out, int max, int* count) {
    QE_API_BEGIN
    check_state(s);
    if (!count || (max > 0 && !out)) fail(QE_ERR_ARG, "NULL output");
    flush(s);
    QE_CUDA(cudaStreamSynchronize(s->stream));
    std::vector<std::string> names;
    std::vector<qe_kernel_profile> acc;
    for (auto& r : s->prof) {
        float ms = 0.f;
        QE_CUDA(cudaEventElapsedTime(&ms, r.start, r.stop));
        size_t i = std::find(names.begin(), names.end(), std::string(r.tag)) - names.begin();
        if (i == names.size()) {
            names.push_back(r.tag);
            qe_kernel_profile p{};
            std::strncpy(p.name, r.tag, sizeof(p.name) - 1);
            acc.push_back(p);
        }
        acc[i].launches += 1;
        acc[i].total_ms += ms;
        acc[i].bytes += r.bytes;
    }
    *count = (int)acc.size();
    for (int i = 0; i < (int)acc.size() && i < max; ++i) out[i] = acc[i];
    QE_API_END
}

int qe_batch_create(int count, const int* nqubits, int layers, const double* angles, double hx,
                    int dtype, void* stream, qe_batch** out) {
    QE_API_BEGIN
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !nqubits || !angles || layers < 1) fail(QE_ERR_ARG, "bad batch description");
    if (dtype != QE_C64 && dtype != QE_C128) fail(QE_ERR_ARG, "unknown dtype");
    if (!std::isfinite(hx)) fail(QE_ERR_ARG, "non-finite field");
    const int nmax = dtype == QE_C64 ? 25 : 23;
    size_t nang = 0;
    for (int c = 0; c < count; ++c) {
        if (nqubits[c] < 1 || nqubits[c] > nmax) fail(QE_ERR_ARG, "qubit count out of range");
        nang += (size_t)2 * layers * nqubits[c];
    }
    for (size_t i = 0; i < nang; ++i)
        if (!std::isfinite(angles[i])) fail(QE_ERR_ARG, "non-finite angle");
    auto* b = new qe_batch();
    b->count = count;
    b->layers = layers;
    b->dtype = dtype;
    b->hx = hx;
    b->stream = (cudaStream_t)stream;
    b->n.assign(nqubits, nqubits + count);
    b->angles.assign(angles, angles + nang);
    b->plan.T = dtype == QE_C64 ? 13 : 12;
    int nbig = 0;
    for (int v : b->n) nbig = std::max(nbig, v);
    while (2 * b->plan.T - 1 < nbig) ++b->plan.T;   // cannot happen within the limits above
    try {
        batch_create(b);
    } catch (...) {
        batch_destroy(b);
        delete b;
        throw;
    }
    *out = b;
    QE_API_END
}

int qe_batch_run(qe_batch* b, double* energies) {
    QE_API_BEGIN
    check_batch(b);
    batch_run(b, energies);
    QE_API_END
}

int qe_batch_set_plan(qe_batch* b, int tile_bits, int tiles_per_item, int threads) {
    QE_API_BEGIN
    check_batch(b);
    batch_set_plan(b, tile_bits, tiles_per_item, threads);
    QE_API_END
}

int qe_batch_set_arith(qe_batch* b, int arith) {
    QE_API_BEGIN
    check_batch(b);
    if (arith != QE_ARITH_FP64 && arith != QE_ARITH_DF64) fail(QE_ERR_ARG, "arith must be QE_ARITH_FP64 or QE_ARITH_DF64");
    batch_set_arith(b, arith);
    QE_API_END
}

int qe_batch_tune(qe_batch* b, int reps, int* tile_bits, int* tiles_per_item, int* threads) {
    QE_API_BEGIN
    check_batch(b);
    if (reps < 1) fail(QE_ERR_ARG, "reps must be >= 1");
    const int tmax = b->dtype == QE_C64 ? 13 : 12;
    int nmax = 0;
    for (int v : b->n) nmax = std::max(nmax, v);
    float best = 1e30f;
    int bt = b->plan.T, bp = b->plan.tiles_per_item, bth = b->plan.threads;
    cudaEvent_t e0, e1;
    QE_CUDA(cudaEventCreate(&e0));
    QE_CUDA(cudaEventCreate(&e1));
    for (int T = tmax - 1; T <= tmax; ++T) {
        if (2 * T - 1 < nmax) continue;
        for (int per : {1, 4, 16})
            for (int th : {128, 256, 512}) {
                batch_set_plan(b, T, per, th);
                batch_run(b, nullptr);   // warm-up
                QE_CUDA(cudaEventRecord(e0, b->stream));
                for (int r = 0; r < reps; ++r) QE_CUDA(cudaGraphLaunch(b->exec, b->stream));
                QE_CUDA(cudaEventRecord(e1, b->stream));
                QE_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                QE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (*b->host_status != 0) fail(QE_ERR_TIMEOUT, "a batch work item timed out while tuning");
                if (ms < best) { best = ms; bt = T; bp = per; bth = th; }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch_set_plan(b, bt, bp, bth);
    if (tile_bits) *tile_bits = bt;
    if (tiles_per_item) *tiles_per_item = bp;
    if (threads) *threads = bth;
    QE_API_END
}

int qe_batch_info(const qe_batch* b, double* hbm_bytes, int* items) {
    QE_API_BEGIN
    check_batch(b);
    if (hbm_bytes) *hbm_bytes = b->hbm_bytes;
    if (items) *items = b->nitems;
    QE_API_END
}

int qe_batch_free(qe_batch* b) {
    QE_API_BEGIN
    if (!b) return QE_OK;
    check_batch(b);
    cudaStreamSynchronize(b->stream);
    batch_destroy(b);
    b->magic = 0;
    delete b;
    QE_API_END
}

static void check_model(const qe_cost_model* m) {
    if (!m || m->magic != 0xC057) fail(QE_ERR_STATE, "invalid cost model handle");
}

int qe_cost_model_create(int hidden1, int hidden2, uint64_t seed, qe_cost_model** out) {
    QE_API_BEGIN
    if (!out) fail(QE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (hidden1 < 1 || hidden1 > 256 || hidden2 < 1 || hidden2 > 256) fail(QE_ERR_ARG, "hidden sizes in [1, 256]");
    auto* m = new qe_cost_model();
    m->d = kCostFeatures;
    m->h1 = hidden1;
    m->h2 = hidden2;
    try {
        mlp_create(m, seed);
    } catch (...) {
        mlp_destroy(m);
        delete m;
        throw;
    }
    *out = m;
    QE_API_END
}

int qe_cost_model_param_count(const qe_cost_model* m, int* count) {
    QE_API_BEGIN
    check_model(m);
    if (!count) fail(QE_ERR_ARG, "count is NULL");
    *count = m->np;
    QE_API_END
}

int qe_cost_model_get_params(const qe_cost_model* m, float* params, int count) {
    QE_API_BEGIN
    check_model(m);
    if (!params || count != m->np) fail(QE_ERR_ARG, "params must hold exactly the parameter count");
    QE_CUDA(cudaStreamSynchronize(m->stream));
    QE_CUDA(cudaMemcpy(params, m->params, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
    QE_API_END
}

int qe_cost_model_set_params(qe_cost_model* m, const float* params, int count) {
    QE_API_BEGIN
    check_model(m);
    if (!params || count != m->np) fail(QE_ERR_ARG, "params must hold exactly the parameter count");
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(params[i])) fail(QE_ERR_ARG, "non-finite parameter");
    QE_CUDA(cudaStreamSynchronize(m->stream));
    QE_CUDA(cudaMemcpy(m->params, params, sizeof(float) * m->np, cudaMemcpyHostToDevice));
    QE_CUDA(cudaMemset(m->mom1, 0, sizeof(float) * m->np));
    QE_CUDA(cudaMemset(m->mom2, 0, sizeof(float) * m->np));
    m->step = 0;
    QE_API_END
}

static void check_samples(const float* X, const float* t, int n) {
    if (n < 1 || !X) fail(QE_ERR_ARG, "need n >= 1 samples");
    for (long i = 0; i < (long)n * kCostFeatures; ++i)
        if (!std::isfinite(X[i])) fail(QE_ERR_ARG, "non-finite feature");
    if (t)
        for (int i = 0; i < n; ++i)
            if (!std::isfinite(t[i])) fail(QE_ERR_ARG, "non-finite target");
}

int qe_cost_model_gradient(qe_cost_model* m, const float* X, const float* t, int n, float* grad,
                           float* loss) {
    QE_API_BEGIN
    check_model(m);
    check_samples(X, t, n);
    if (!t || !grad) fail(QE_ERR_ARG, "targets and grad are required");
    const float l = mlp_gradient(m, X, t, n, grad);
    if (loss) *loss = l;
    QE_API_END
}

int qe_cost_model_train(qe_cost_model* m, const float* X, const float* t, int n, int epochs,
                        float lr, float* loss) {
    QE_API_BEGIN
    check_model(m);
    check_samples(X, t, n);
    if (!t || epochs < 0 || !(lr > 0.f)) fail(QE_ERR_ARG, "bad training arguments");
    const float l = mlp_train(m, X, t, n, epochs, lr);
    if (loss) *loss = l;
    QE_API_END
}

int qe_cost_model_predict(qe_cost_model* m, const float* X, int n, float* y) {
    QE_API_BEGIN
    check_model(m);
    check_samples(X, nullptr, n);
    if (!y) fail(QE_ERR_ARG, "y is NULL");
    mlp_predict(m, X, n, y);
    QE_API_END
}

int qe_cost_model_free(qe_cost_model* m) {
    QE_API_BEGIN
    if (!m) return QE_OK;
    check_model(m);
    mlp_destroy(m);
    m->magic = 0;
    delete m;
    QE_API_END
}

int qe_cost_features(int op, int n, int dtype, int k, int lo, int hi, int m, uint64_t c, float* f) {
    QE_API_BEGIN
    if (!f || op < 0 || op > 4 || n < 1 || n > 34) fail(QE_ERR_ARG, "bad feature request");
    cost_features(op, n, dtype, k, lo, hi, m, c, f);
    QE_API_END
}

int qe_set_cost_model(qe_state* s, qe_cost_model* model) {
    QE_API_BEGIN
    check_state(s);
    if (model) check_model(model);
    flush(s);
    s->model = model;
    QE_API_END
}

int qe_planned_fusion_width(qe_state* s, int* k) {
    QE_API_BEGIN
    check_state(s);
    if (!k) fail(QE_ERR_ARG, "k is NULL");
    *k = choose_fusion_width(s, s->queue);
    QE_API_END
}

int qe_reset_stats(qe_state* s) {
    QE_API_BEGIN
    check_state(s);
    s->stats = Stats();
    QE_API_END
}

}  // extern "C"

// Batched correction steps of many flow instances (serving).
//
// The correction step of Algorithm 2 is per instance; its network (Eq. gru + output
// layer) works patch by patch with weights shared by every instance that uses
// the same net.  A server therefore runs one step of several instances as:
//   per instance  S1+S2+S3 into that instance's rows of one feature matrix X,
//   once          S4 over all rows of X (one tensor-core GRU launch),
//   per instance  S5, S6, S7 from that instance's rows of d.
// Each instance's GRU state h lives in a segment of one state pool.  Segments
// and batch rows are whole 128-row tiles, so every GRU tile belongs to one
// instance; a per-tile table gives the tile's first state row in the pool.
// A patch row's arithmetic does not depend on the other rows of its tile, so
// an instance gets the same bits alone (dnnmg_step) and in any batch.  The
// per-instance passes of up to kLanes instances run side by side on the
// server's own streams (small meshes fill few SMs each), each stream with its
// own scratch; the caller's stream forks to them and joins back around S4.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"

namespace dnnmg {
namespace {

constexpr int kTileRows = 128;   // rows of one GRU tile
constexpr int kLanes = 8;        // side streams: the per-instance passes of up to 8 instances overlap

// First-fit allocator of row ranges in units of `unit` rows; frees coalesce.
struct RowPool {
    int capacity = 0, unit = 1;
    std::map<int, int> free_;   // start -> length, disjoint, never adjacent
    std::map<int, int> used_;   // start -> length

    void init(int cap, int u) {
        unit = u;
        capacity = cap / u * u;
        free_.clear();
        used_.clear();
        if (capacity > 0) free_[0] = capacity;
    }
    int rounded(int rows) const { return (rows + unit - 1) / unit * unit; }
    // start of a free range of rounded(rows) rows, or -1
    int alloc(int rows) {
        const int n = rounded(rows);
        if (n <= 0) return -1;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const int start = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[start + n] = len - n;
            used_[start] = n;
            return start;
        }
        return -1;
    }
    bool release(int start) {
        auto u = used_.find(start);
        if (u == used_.end()) return false;
        int s = start, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(s);
        if (next != free_.end() && next->first == s + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == s) {
                s = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[s] = len;
        return true;
    }
    int used_rows() const {
        int n = 0;
        for (auto &kv : used_) n += kv.second;
        return n;
    }
    int largest_free() const {
        int m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

}  // namespace
}  // namespace dnnmg

struct dnnmg_pool_s {
    dnnmg::RowPool pool;
};

struct dnnmg_server_s {
    dnnmg_net_t net = nullptr;
    int device = -1;
    int cap_rows = 0;
    dnnmg::RowPool pool;
    float *hpool = nullptr;   // [cap_rows][H]
    void *X = nullptr;        // [cap_rows][ldx] bf16
    float *d = nullptr;       // [cap_rows][n_out]
    int *tiles_dev = nullptr; // [cap_rows / 128]
    int *tiles_host[2] = {nullptr, nullptr};   // pinned staging, used in turn
    cudaEvent_t tiles_ev[2] = {nullptr, nullptr};
    int flip = 0;
    // per side stream: v_corr and the padded x_c of the largest admitted mesh
    cudaStream_t lane[dnnmg::kLanes] = {};
    cudaEvent_t lane_done[dnnmg::kLanes] = {};
    cudaEvent_t fork = nullptr;
    void *scratch[dnnmg::kLanes] = {};
    size_t scratch_bytes = 0;
    struct Slot {
        dnnmg_mesh_t mesh;
        int start, rows;      // pool segment (multiple of 128 rows); rows = padded patch rows
        bool live;
    };
    std::vector<Slot> slots;
};

namespace dnnmg {
namespace {

size_t scratch_need(const dnnmg_mesh_info &I) {
    return align256(2 * (size_t)I.plane * I.real_bytes) +
           align256(3 * (size_t)(I.nyc + 1) * round_up(I.nxc + 1, 32) * I.real_bytes);
}

void server_free(dnnmg_server_s *s) {
    if (!s) return;
    cudaFree(s->hpool);
    cudaFree(s->X);
    cudaFree(s->d);
    cudaFree(s->tiles_dev);
    for (int j = 0; j < kLanes; ++j) {
        cudaFree(s->scratch[j]);
        if (s->lane[j]) cudaStreamDestroy(s->lane[j]);
        if (s->lane_done[j]) cudaEventDestroy(s->lane_done[j]);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    for (int b = 0; b < 2; ++b) {
        if (s->tiles_host[b]) cudaFreeHost(s->tiles_host[b]);
        if (s->tiles_ev[b]) cudaEventDestroy(s->tiles_ev[b]);
    }
    delete s;
}

int check_server(dnnmg_server_s *s) {
    if (!s) return fail(DNNMG_EINVAL, "server handle is NULL");
    int cur = -1;
    DNNMG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != s->device) return fail(DNNMG_EINVAL, "server belongs to device %d but device %d is current", s->device, cur);
    return DNNMG_OK;
}

int check_slot(dnnmg_server_s *s, int slot) {
    if (slot < 0 || slot >= (int)s->slots.size() || !s->slots[slot].live)
        return fail(DNNMG_EINVAL, "slot %d is not an admitted instance", slot);
    return DNNMG_OK;
}

}  // namespace
}  // namespace dnnmg

using namespace dnnmg;

extern "C" {

int dnnmg_pool_create(int capacity_rows, int unit, dnnmg_pool_t *out) {
    clear_error();
    if (!out) return fail(DNNMG_EINVAL, "out is NULL");
    if (capacity_rows < 0 || unit < 1) return fail(DNNMG_EINVAL, "capacity %d / unit %d", capacity_rows, unit);
    dnnmg_pool_s *p = new (std::nothrow) dnnmg_pool_s();
    if (!p) return fail(DNNMG_ENOMEM, "host allocation failed");
    p->pool.init(capacity_rows, unit);
    *out = p;
    return DNNMG_OK;
}

int dnnmg_pool_alloc(dnnmg_pool_t pool, int rows, int *start) {
    clear_error();
    if (!pool || !start) return fail(DNNMG_EINVAL, "NULL argument");
    if (rows < 1) return fail(DNNMG_EINVAL, "rows = %d", rows);
    const int s = pool->pool.alloc(rows);
    if (s < 0) return fail(DNNMG_ENOMEM, "no free range of %d rows", pool->pool.rounded(rows));
    *start = s;
    return DNNMG_OK;
}

int dnnmg_pool_free(dnnmg_pool_t pool, int start) {
    clear_error();
    if (!pool) return fail(DNNMG_EINVAL, "pool is NULL");
    if (!pool->pool.release(start)) return fail(DNNMG_EINVAL, "no range starts at row %d", start);
    return DNNMG_OK;
}

int dnnmg_pool_stats(dnnmg_pool_t pool, int *used_rows, int *largest_free) {
    clear_error();
    if (!pool) return fail(DNNMG_EINVAL, "pool is NULL");
    if (used_rows) *used_rows = pool->pool.used_rows();
    if (largest_free) *largest_free = pool->pool.largest_free();
    return DNNMG_OK;
}

void dnnmg_pool_destroy(dnnmg_pool_t pool) { delete pool; }

size_t dnnmg_server_bytes(dnnmg_net_t net, int max_rows) {
    if (!net || max_rows < 0) return 0;
    const size_t rows = (size_t)(max_rows + kTileRows - 1) / kTileRows * kTileRows;
    return align256(rows * net->H * sizeof(float)) + align256(rows * net->ldx * 2) +
           align256(rows * net->n_out * sizeof(float)) + align256(rows / kTileRows * sizeof(int));
}

int dnnmg_server_create(dnnmg_net_t net, int max_rows, dnnmg_server_t *out) {
    clear_error();
    if (!out) return fail(DNNMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!net) return fail(DNNMG_EINVAL, "net handle is NULL");
    if (!net->tc)
        return fail(DNNMG_EUNSUPPORTED, "batched steps need a tensor-core (DNNMG_BF16NET, H <= 128) network");
    if (max_rows < 1) return fail(DNNMG_EINVAL, "max_rows = %d", max_rows);
    int dev = -1;
    DNNMG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != net->device) return fail(DNNMG_EINVAL, "net belongs to device %d but device %d is current", net->device, dev);
    dnnmg_server_s *s = new (std::nothrow) dnnmg_server_s();
    if (!s) return fail(DNNMG_ENOMEM, "host allocation failed");
    s->net = net;
    s->device = dev;
    s->cap_rows = (max_rows + kTileRows - 1) / kTileRows * kTileRows;
    s->pool.init(s->cap_rows, kTileRows);
    const size_t rows = (size_t)s->cap_rows, ntiles = rows / kTileRows;
    bool ok = cudaMalloc(&s->hpool, rows * net->H * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&s->X, rows * net->ldx * 2) == cudaSuccess &&
              cudaMalloc(&s->d, rows * net->n_out * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&s->tiles_dev, ntiles * sizeof(int)) == cudaSuccess;
    for (int b = 0; ok && b < 2; ++b)
        ok = cudaMallocHost(&s->tiles_host[b], ntiles * sizeof(int)) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->tiles_ev[b], cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; ok && j < kLanes; ++j)
        ok = cudaStreamCreateWithFlags(&s->lane[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->lane_done[j], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) == cudaSuccess;
    // feature rows past an instance's patches are read by its last GRU tile:
    // keep them finite (their results land only in the instance's padding)
    ok = ok && cudaMemset(s->X, 0, rows * net->ldx * 2) == cudaSuccess;
    if (!ok) {
        server_free(s);
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the server's %zu bytes failed", dnnmg_server_bytes(net, max_rows));
    }
    *out = s;
    return DNNMG_OK;
}

int dnnmg_server_destroy(dnnmg_server_t server) {
    clear_error();
    if (!server) return DNNMG_OK;
    cudaDeviceSynchronize();
    server_free(server);
    return DNNMG_OK;
}

int dnnmg_server_admit(dnnmg_server_t s, dnnmg_mesh_t mesh, int *slot) {
    clear_error();
    if (int e = check_server(s)) return e;
    if (!mesh || !slot) return fail(DNNMG_EINVAL, "NULL argument");
    if (mesh->device != s->device) return fail(DNNMG_EINVAL, "mesh and server are on different devices");
    const dnnmg_mesh_info &I = mesh->info;
    const Net &n = *s->net;
    if (I.precision != DNNMG_BF16NET) return fail(DNNMG_EINVAL, "mesh precision must be DNNMG_BF16NET");
    if (I.n_in != n.n_in || I.ldx != n.ldx || I.n_out != n.n_out)
        return fail(DNNMG_EINVAL, "mesh has n_in %d / n_out %d, the net %d / %d", I.n_in, I.n_out, n.n_in, n.n_out);
    const int rows = (I.P + kTileRows - 1) / kTileRows * kTileRows;
    int start = 0;
    if (rows > 0) {
        start = s->pool.alloc(rows);
        if (start < 0)
            return fail(DNNMG_ENOMEM, "no free state segment of %d rows (largest %d of %d)", rows,
                        s->pool.largest_free(), s->cap_rows);
    }
    const size_t need = scratch_need(I);
    if (need > s->scratch_bytes) {
        // the scratch may be in use by steps in flight
        cudaError_t e = cudaDeviceSynchronize();
        void *p[kLanes] = {};
        for (int j = 0; e == cudaSuccess && j < kLanes; ++j) e = cudaMalloc(&p[j], need);
        if (e != cudaSuccess) {
            for (int j = 0; j < kLanes; ++j) cudaFree(p[j]);
            if (rows > 0) s->pool.release(start);
            cudaGetLastError();
            return fail(DNNMG_ENOMEM, "scratch of %d x %zu bytes: %s", kLanes, need, cudaGetErrorString(e));
        }
        for (int j = 0; j < kLanes; ++j) {
            cudaFree(s->scratch[j]);
            s->scratch[j] = p[j];
        }
        s->scratch_bytes = need;
    }
    // h0 = 0 (Sec. 6.2), padding rows included
    if (rows > 0 && cudaMemset(s->hpool + (size_t)start * n.H, 0, (size_t)rows * n.H * sizeof(float)) != cudaSuccess) {
        s->pool.release(start);
        cudaGetLastError();
        return fail(DNNMG_ECUDA, "clearing the state segment failed");
    }
    int id = -1;
    for (int i = 0; i < (int)s->slots.size(); ++i)
        if (!s->slots[i].live) {
            id = i;
            break;
        }
    if (id < 0) {
        id = (int)s->slots.size();
        s->slots.push_back({});
    }
    s->slots[id] = {mesh, start, rows, true};
    *slot = id;
    return DNNMG_OK;
}

int dnnmg_server_release(dnnmg_server_t s, int slot) {
    clear_error();
    if (int e = check_server(s)) return e;
    if (int e = check_slot(s, slot)) return e;
    // a step in flight may still read or write the segment
    DNNMG_CUDA_TRY(cudaDeviceSynchronize());
    if (s->slots[slot].rows > 0) s->pool.release(s->slots[slot].start);
    s->slots[slot].live = false;
    s->slots[slot].mesh = nullptr;
    return DNNMG_OK;
}

int dnnmg_server_state(dnnmg_server_t s, int slot, float **h) {
    clear_error();
    if (!s) return fail(DNNMG_EINVAL, "server handle is NULL");
    if (int e = check_slot(s, slot)) return e;
    if (!h) return fail(DNNMG_EINVAL, "h is NULL");
    *h = s->hpool + (size_t)s->slots[slot].start * s->net->H;
    return DNNMG_OK;
}

int dnnmg_server_step(dnnmg_server_t s, int n, const int *slots, const double *const *xc, void *const *bf,
                      double *const *bc, const double *t, cudaStream_t stream) {
    clear_error();
    if (int e = check_server(s)) return e;
    if (n < 1 || !slots || !xc || !bf || !bc || !t) return fail(DNNMG_EINVAL, "empty batch or NULL argument");
    std::vector<int> row0(n);
    int total = 0;
    for (int i = 0; i < n; ++i) {
        if (int e = check_slot(s, slots[i])) return e;
        for (int j = 0; j < i; ++j)
            if (slots[j] == slots[i]) return fail(DNNMG_EINVAL, "slot %d appears twice in one batch", slots[i]);
        if (!xc[i] || !bf[i] || !bc[i]) return fail(DNNMG_EINVAL, "NULL array of instance %d", i);
        if (reinterpret_cast<uintptr_t>(bf[i]) % 16) return fail(DNNMG_EINVAL, "bf of instance %d is not 16-byte aligned", i);
        row0[i] = total;
        total += s->slots[slots[i]].rows;
    }
    // per tile of the batch: its first state row in the pool
    const int b = s->flip;
    s->flip ^= 1;
    DNNMG_CUDA_TRY(cudaEventSynchronize(s->tiles_ev[b]));   // the staging buffer's last copy has been read
    int *tiles = s->tiles_host[b];
    for (int i = 0; i < n; ++i) {
        const dnnmg_server_s::Slot &sl = s->slots[slots[i]];
        for (int k = 0; k < sl.rows / kTileRows; ++k) tiles[row0[i] / kTileRows + k] = sl.start + k * kTileRows;
    }
    const Net &net = *s->net;
    if (total > 0) {
        DNNMG_CUDA_TRY(cudaMemcpyAsync(s->tiles_dev, tiles, (size_t)(total / kTileRows) * sizeof(int),
                                       cudaMemcpyHostToDevice, stream));
        DNNMG_CUDA_TRY(cudaEventRecord(s->tiles_ev[b], stream));
    }
    // the per-instance passes go round-robin to the side streams, which fork
    // from and join back into the caller's stream around each phase
    const int nl = n < kLanes ? n : kLanes;
    auto fork = [&]() -> int {
        DNNMG_CUDA_TRY(cudaEventRecord(s->fork, stream));
        for (int j = 0; j < nl; ++j) DNNMG_CUDA_TRY(cudaStreamWaitEvent(s->lane[j], s->fork, 0));
        return DNNMG_OK;
    };
    auto join = [&]() -> int {
        for (int j = 0; j < nl; ++j) {
            DNNMG_CUDA_TRY(cudaEventRecord(s->lane_done[j], s->lane[j]));
            DNNMG_CUDA_TRY(cudaStreamWaitEvent(stream, s->lane_done[j], 0));
        }
        return DNNMG_OK;
    };
    uint16_t *X = static_cast<uint16_t *>(s->X);
    // S1 + S2 + S3 per instance, into its rows of X
    if (int e = fork()) return e;
    for (int i = 0; i < n; ++i) {
        const dnnmg_mesh_s &m = *s->slots[slots[i]].mesh;
        const dnnmg_mesh_info &I = m.info;
        cudaStream_t st = s->lane[i % kLanes];
        void *xcp = static_cast<char *>(s->scratch[i % kLanes]) + align256(2 * (size_t)I.plane * I.real_bytes);
        DNNMG_CUDA_TRY(launch_coarse_pad(m.g, I.precision, xc[i], xcp, st));
        // the same two S2+S3 kernels as dnnmg_step, so an instance gets the same bits
        void *Xi = X + (size_t)row0[i] * net.ldx;
        const bool cf = residual_cf_supported(m.g, I.precision);
        if (cf) DNNMG_CUDA_TRY(launch_residual_cf(m.g, I.precision, m.fem32, xcp, bf[i], Xi, st));
        DNNMG_CUDA_TRY(launch_residual_step(m.g, I.precision, m.fem64, m.fem32, xcp, t[i], bf[i], Xi, st, cf));
    }
    if (int e = join()) return e;
    // S4 once over every instance's rows
    if (total > 0)
        DNNMG_CUDA_TRY(launch_gru_tc_rows(net, s->X, s->hpool, s->d, total, s->tiles_dev, s->cap_rows, stream));
    // S5, S6, S7 per instance, from its rows of d
    if (int e = fork()) return e;
    for (int i = 0; i < n; ++i) {
        const dnnmg_mesh_s &m = *s->slots[slots[i]].mesh;
        const dnnmg_mesh_info &I = m.info;
        cudaStream_t st = s->lane[i % kLanes];
        void *vc = s->scratch[i % kLanes];
        const float *d = s->d + (size_t)row0[i] * net.n_out;
        DNNMG_CUDA_TRY(launch_scatter_avg(m.g, I.precision, d, nullptr, xc[i], t[i], vc, st));
        DNNMG_CUDA_TRY(launch_rhs(m.g, I.precision, m.fem64, m.fem32, vc, bf[i], st));
        DNNMG_CUDA_TRY(launch_restrict(m.g, I.precision, bf[i], bc[i], st));
    }
    if (int e = join()) return e;
    return DNNMG_OK;
}

}  // extern "C"

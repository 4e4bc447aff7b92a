// Host side of the batched kernel: table deduplication, cost-balanced
// segment schedule, descriptor upload and the per-stage launch.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "dispatch.cuh"

namespace gpweno {

// Relative cost of one face for radius R (the scheme's operation count per face,
// normalised to R = 2; see costmodel.py).
inline double face_cost(int R) { return R == 1 ? 0.61 : (R == 2 ? 1.0 : 1.59); }

struct BatchInstInfo {
    int nx, ny, R, W, nstrips;
    double row_cost, warm_cost;
};

// Greedy contiguous partition of the (instance, strip, row) work list into
// at most `grid` CTA shares of roughly equal estimated cost.  Returns the
// number of CTAs used; fills segments and per-CTA start offsets.
inline int partition_batch(const std::vector<BatchInstInfo> &info, const std::vector<int> &order, int grid,
                           double budget, std::vector<BatchSeg> &segs, std::vector<int> &start, int min_rows = 8)
{
    segs.clear();
    start.assign(1, 0);
    double left = budget;
    for (int oi : order) {
        const BatchInstInfo &I = info[oi];
        for (int st = 0; st < I.nstrips; ++st) {
            int y = 0;
            while (y < I.ny) {
                // rows affordable in this CTA after paying the segment warm-up
                double avail = left - I.warm_cost;
                int rows = avail > 0 ? (int)std::floor(avail / I.row_cost) : 0;
                if (rows < 1 || (rows < min_rows && I.ny - y > rows)) {
                    if (left < budget) {       // close this CTA and open a fresh one
                        start.push_back((int)segs.size());
                        left = budget;
                        continue;
                    }
                    rows = std::max(1, rows);  // a single segment larger than a budget
                }
                rows = std::min(rows, I.ny - y);
                segs.push_back({oi, st, y, y + rows});
                left -= I.warm_cost + rows * I.row_cost;
                y += rows;
            }
        }
    }
    if ((int)segs.size() > start.back()) start.push_back((int)segs.size());
    return (int)start.size() - 1;
}

inline unsigned long long batch_hash(const std::vector<BatchInstInfo> &info)
{
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](unsigned long long v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    for (const auto &I : info) {
        mix((unsigned long long)I.nx);
        mix((unsigned long long)I.ny);
        mix((unsigned long long)I.R);
    }
    return h;
}

// Schedule parameters of a batch: block size, resident CTAs per SM, the cap on a
// strip's width (columns), the fewest rows a segment may have when it does not
// finish its strip, and CTA shares per resident slot.
struct BatchTiles {
    int nt = 0, cps = 0, wcap = 0, min_rows = 8, oversub = 1;
};

// Tuning cache: text lines "<signature hex> <block> <ctas_per_sm> [<strip width cap>
// <min segment rows> <CTA shares per slot>]" (0 for the width cap: the block allows).
inline bool read_tune_cache(const char *path, unsigned long long sig, BatchTiles &t)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long s;
        int a, b, w = 0, r = 8, o = 1;
        const int got = std::sscanf(line, "%llx %d %d %d %d %d", &s, &a, &b, &w, &r, &o);
        if ((got == 3 || got == 6) && s == sig && (a == 128 || a == 256) && b >= 1 && b <= 8 && w >= 0 &&
            (w == 0 || w >= 16) && r >= 1 && r <= 1024 && o >= 1 && o <= 16) {
            t.nt = a;
            t.cps = b;
            t.wcap = w;
            t.min_rows = r;
            t.oversub = o;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

template <typename T, int NT>
gpweno_status batch_occupancy(int &occ)
{
    auto kern = batch_stage_kernel<T, NT>;
    const size_t smem = batch_smem_bytes<T, NT>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "batch smem attribute");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
    if (e != cudaSuccess) return cuda_fail(e, "batch occupancy");
    if (occ < 1) {
        set_error("batch kernel cannot be resident");
        return GPWENO_ERR_CUDA;
    }
    return GPWENO_OK;
}

template <typename T>
gpweno_status build_batch_T(gpweno_plan b)
{
    const int n = (int)b->members.size();
    // ---- deduplicate table sets per radius --------------------------------
    BatchTables<T> bt;
    std::memset(&bt, 0, sizeof(bt));
    std::vector<gpweno_plan> reps[4];
    b->member_tab.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        gpweno_plan p = b->members[k];
        auto &rv = reps[p->R];
        int idx = -1;
        for (int q = 0; q < (int)rv.size(); ++q)
            if (rv[q]->ell == p->ell && rv[q]->opts.sigma_over_dx == p->opts.sigma_over_dx &&
                rv[q]->gamma == p->gamma && rv[q]->opts.eps == p->opts.eps && rv[q]->opts.p == p->opts.p &&
                rv[q]->opts.flux_form == p->opts.flux_form && rv[q]->opts.candidates == p->opts.candidates)
                idx = q;
        if (idx < 0) {
            if ((int)rv.size() >= kBatchMaxSets) {
                set_error("gpweno_plan_batch: more than %d distinct (l, sigma, gamma, eps, p) sets for R=%d",
                          kBatchMaxSets, p->R);
                return GPWENO_ERR_ARG;
            }
            idx = (int)rv.size();
            rv.push_back(p);
            if (p->R == 1) bt.t1[idx] = make_tables<T, 1>(p);
            if (p->R == 2) bt.t2[idx] = make_tables<T, 2>(p);
            if (p->R == 3) bt.t3[idx] = make_tables<T, 3>(p);
        }
        b->member_tab[k] = idx;
    }
    b->batch_tables.assign(reinterpret_cast<unsigned char *>(&bt), reinterpret_cast<unsigned char *>(&bt) + sizeof(bt));

    // ---- schedule -----------------------------------------------------------
    std::vector<BatchInstInfo> info(n);
    for (int k = 0; k < n; ++k) {
        gpweno_plan p = b->members[k];
        BatchInstInfo &I = info[k];
        I.nx = p->dims.n[0];
        I.ny = p->dims.n[1];
        I.R = p->R;
    }
    b->batch_signature = batch_hash(info);
    BatchTiles tiles;
    if (!read_tune_cache(b->batch_tune_path.empty() ? nullptr : b->batch_tune_path.c_str(), b->batch_signature,
                         tiles)) {
        // built-in choice: narrow instances waste most lanes of a 256-thread strip
        std::vector<int> widths;
        for (const auto &I : info) widths.push_back(I.nx);
        std::nth_element(widths.begin(), widths.begin() + n / 2, widths.end());
        tiles.nt = widths[n / 2] < 400 ? 128 : 256;
        tiles.cps = 0;   // occupancy limit
        // several CTA shares per resident slot: the hardware scheduler then evens out what
        // the cost estimate misses (one share per slot measured 1.9x slower on a 256-instance
        // batch; 8 to 16 shares all came within 2 % of the best)
        tiles.oversub = 8;
    }
    const int nt = tiles.nt;
    int cps = tiles.cps;
    int occ = 0;
    gpweno_status s = nt == 128 ? batch_occupancy<T, 128>(occ) : batch_occupancy<T, 256>(occ);
    if (s != GPWENO_OK) return s;
    if (cps <= 0 || cps > occ) cps = occ;
    b->batch_nt = nt;
    b->batch_ctas_per_sm = cps;
    const int wmax = tiles.wcap > 0 ? std::min(nt - 5, tiles.wcap) : nt - 5;
    b->batch_wcap = wmax;
    b->batch_min_rows = tiles.min_rows;
    b->batch_oversub = tiles.oversub;
    double total = 0.0;
    for (auto &I : info) {
        I.nstrips = (I.nx + wmax - 1) / wmax;
        I.W = (I.nx + I.nstrips - 1) / I.nstrips;
        const double wx = std::ceil((I.W + 5) / 32.0), wy = std::ceil(I.W / 32.0);
        I.row_cost = (wx + wy) * face_cost(I.R) + 0.15 * wy;
        I.warm_cost = 5.0 * wy * face_cost(I.R) + (2 * I.R + 2) * 0.05 * wy;
        total += I.nstrips * (I.ny * I.row_cost + I.warm_cost);
    }
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return info[x].R > info[y].R; });
    const int grid = cps * b->num_sms * tiles.oversub;
    std::vector<BatchSeg> segs;
    std::vector<int> start;
    double budget = total / grid;
    int used = partition_batch(info, order, grid, budget, segs, start, tiles.min_rows);
    for (int it = 0; it < 60 && used > grid; ++it) {
        budget *= 1.01;
        used = partition_batch(info, order, grid, budget, segs, start, tiles.min_rows);
    }
    b->batch_grid = used;
    b->batch_nseg = (int)segs.size();

    // ---- device arrays --------------------------------------------------------
    cudaError_t e;
    if ((e = cudaMalloc(&b->batch_inst_dev, sizeof(BatchInst<T>) * n)) != cudaSuccess)
        return cuda_fail(e, "batch descriptors");
    if ((e = cudaMallocHost(&b->batch_inst_host, sizeof(BatchInst<T>) * n)) != cudaSuccess)
        return cuda_fail(e, "batch descriptor staging");
    if ((e = cudaMalloc(&b->batch_segs_dev, sizeof(BatchSeg) * segs.size())) != cudaSuccess)
        return cuda_fail(e, "batch segments");
    if ((e = cudaMalloc(&b->batch_cta_dev, sizeof(int) * start.size())) != cudaSuccess)
        return cuda_fail(e, "batch CTA offsets");
    if ((e = cudaMemcpy(b->batch_segs_dev, segs.data(), sizeof(BatchSeg) * segs.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "batch segments upload");
    if ((e = cudaMemcpy(b->batch_cta_dev, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "batch CTA offsets upload");
    BatchInst<T> *h = static_cast<BatchInst<T> *>(b->batch_inst_host);
    for (int k = 0; k < n; ++k) {
        gpweno_plan p = b->members[k];
        BatchInst<T> &d = h[k];
        std::memset(&d, 0, sizeof(d));
        d.n[0] = p->dims.n[0];
        d.n[1] = p->dims.n[1];
        d.per[0] = p->dims.bc_lo[0] == GPWENO_BC_PERIODIC;
        d.per[1] = p->dims.bc_lo[1] == GPWENO_BC_PERIODIC;
        d.idx[0] = (T)(1.0 / p->dims.dx[0]);
        d.idx[1] = (T)(1.0 / p->dims.dx[1]);
        d.R = p->R;
        d.tab = b->member_tab[k];
        d.W = info[k].W;
        d.nstrips = info[k].nstrips;
    }
    b->batch_last_ptrs.assign(2 * n, nullptr);
    return GPWENO_OK;
}

template <typename T>
gpweno_status launch_batch_stage_T(gpweno_plan b, int stage, void *const *U, void *const *scratch,
                                   const double *dt_dev, cudaStream_t st)
{
    const int n = (int)b->members.size();
    if (stage == 0) {
        // refresh the buffer pointers of the descriptors when they changed
        bool changed = false;
        BatchInst<T> *h = static_cast<BatchInst<T> *>(b->batch_inst_host);
        for (int k = 0; k < n; ++k) {
            if (b->batch_last_ptrs[2 * k] != U[k] || b->batch_last_ptrs[2 * k + 1] != scratch[k]) changed = true;
        }
        if (changed) {
            // the staging buffer may still feed an earlier asynchronous upload
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "batch descriptor staging");
            for (int k = 0; k < n; ++k) {
                gpweno_plan p = b->members[k];
                const size_t bytes = sizeof(T) * (size_t)(p->dims.ndim + 2) * (size_t)p->ncell;
                char *s = static_cast<char *>(scratch[k]);
                h[k].U = static_cast<const T *>(U[k]);
                h[k].D = reinterpret_cast<T *>(s);
                h[k].V1 = reinterpret_cast<T *>(s + bytes);
                h[k].V2 = reinterpret_cast<T *>(s + 2 * bytes);
                h[k].lo = reinterpret_cast<T *>(s + 3 * bytes);
                b->batch_last_ptrs[2 * k] = U[k];
                b->batch_last_ptrs[2 * k + 1] = scratch[k];
            }
            e = cudaMemcpyAsync(b->batch_inst_dev, h, sizeof(BatchInst<T>) * n, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
        }
    }
    BatchTables<T> bt;
    std::memcpy(&bt, b->batch_tables.data(), sizeof(bt));
    const int *flags = reinterpret_cast<const int *>(b->ws + 3);
    if (b->batch_nt == 128) {
        batch_stage_kernel<T, 128><<<b->batch_grid, 128, batch_smem_bytes<T, 128>(), st>>>(
            static_cast<const BatchInst<T> *>(b->batch_inst_dev), static_cast<const BatchSeg *>(b->batch_segs_dev),
            static_cast<const int *>(b->batch_cta_dev), stage, dt_dev, const_cast<int *>(flags), bt);
    } else {
        batch_stage_kernel<T, 256><<<b->batch_grid, 256, batch_smem_bytes<T, 256>(), st>>>(
            static_cast<const BatchInst<T> *>(b->batch_inst_dev), static_cast<const BatchSeg *>(b->batch_segs_dev),
            static_cast<const int *>(b->batch_cta_dev), stage, dt_dev, const_cast<int *>(flags), bt);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

}  // namespace gpweno

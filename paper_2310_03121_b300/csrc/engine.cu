// Workspaces and the launch sequence of one evaluation.
//
// One evaluation (paper, section "PyTorch Model Support": positions in,
// energy out, forces as the energy gradient) on one stream:
//   stage -> [cell list] -> neighbors -> AEV -> network (+ backward) ->
//   AEV backward (forces) -> finalize (FP64 energies, FP32 forces).
// All device memory of an evaluation is reserved up front in a Workspace;
// nothing is allocated per call.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "engine.cuh"

namespace mlp {

Box make_box(int periodic, const double* L) {
    Box b{};
    b.periodic = periodic;
    for (int a = 0; a < 3; ++a) {
        double l = periodic ? L[a] : 1.0;
        b.L[a] = (float)l;
        b.Lhi[a] = (float)l;
        b.Llo[a] = (float)(l - (double)b.Lhi[a]);
        b.invL[a] = (float)(1.0 / l);
    }
    return b;
}

Grid make_periodic_grid(const double* L, float r_list, long long max_cells) {
    // Cells at least r_list wide: floor(L / r_list) per axis. The product is
    // formed in 64 bits and, where it exceeds max_cells (a large box with a
    // short cutoff), the largest axis loses cells until it fits: wider cells
    // only add candidates to the search, never lose a neighbor.
    long long nc[3];
    for (int a = 0; a < 3; ++a) {
        double f = std::floor(L[a] / (double)r_list);
        nc[a] = f < 1.0 ? 1 : (f > 1048576.0 ? 1048576 : (long long)f);
    }
    if (max_cells < 1) max_cells = 1;
    auto prod = [&]() { return nc[0] * nc[1] * nc[2]; };
    if (prod() > max_cells) {
        const double scale = std::cbrt((double)prod() / (double)max_cells);
        for (int a = 0; a < 3; ++a) nc[a] = std::max(1LL, (long long)std::floor((double)nc[a] / scale));
    }
    while (prod() > max_cells) {
        int big = 0;
        for (int a = 1; a < 3; ++a) if (nc[a] > nc[big]) big = a;
        nc[big] -= 1;
    }
    Grid g{};
    for (int a = 0; a < 3; ++a) {
        g.nc[a] = (int)nc[a];
        g.origin[a] = 0.f;
        g.inv_cs[a] = (float)((double)nc[a] / L[a]);
    }
    g.ncell = (int)prod();
    return g;
}

static int rows_capacity(int cap_atoms) {
    long long r = (long long)cap_atoms + kNSpecies * (kTileRows - 1);
    return (int)(((r + kTileRows - 1) / kTileRows) * kTileRows);
}

namespace {
struct Plan {
    size_t total = 0;
    struct Item {
        void** dst;
        size_t bytes;
    };
    std::vector<Item> items;
    template <typename T>
    void add(T** p, size_t count) {
        size_t b = ((count * sizeof(T)) + 255) / 256 * 256;
        if (b == 0) b = 256;
        items.push_back({reinterpret_cast<void**>(p), b});
        total += b;
    }
};

void plan_workspace(Plan& P, Workspace& ws) {
    const size_t n = ws.cap_atoms, R = ws.rows_cap;
    P.add(&ws.hi, n);
    P.add(&ws.lo, n);
    P.add(&ws.ref, n);
    P.add(&ws.rank, n);
    P.add(&ws.nbr_cnt, n);
    P.add(&ws.nbr, n * (size_t)ws.nbr_cap);
    P.add(&ws.row_atom, R);
    P.add(&ws.ctr, 1);
    P.add(&ws.grad, 3 * n);
    P.add(&ws.e, n * (size_t)ws.e_nets());
    if (ws.precision == 0) {
        P.add(&ws.dG, R * kAevLd);
    } else {
        P.add(&ws.dG16, R * kAevLd);
        if (ws.nets > 1) P.add(&ws.g1ens, R * (size_t)ws.nets * kH1);
    }
    P.add(&ws.ang_big_list, n);
    P.add(&ws.ang_big_flag, n);
    P.add(&ws.tc_err, 4);
    P.add(&ws.err_sticky, 4);
    if (ws.precision == 0) {
        P.add(&ws.G32, R * kAevLd);
        P.add(&ws.fb.Z1, R * kH1);
        P.add(&ws.fb.H1, R * kH1);
        P.add(&ws.fb.Z2, R * kH2);
        P.add(&ws.fb.H2, R * kH2);
        P.add(&ws.fb.H3, R * kH3);
        P.add(&ws.fb.G3, R * kH3);
        P.add(&ws.fb.G2, R * kH2);
        P.add(&ws.fb.G1, R * kH1);
    } else {
        P.add(&ws.G16, R * kAevLd);
        if (ws.precision == 1) P.add(&ws.G16lo, R * kAevLd);
    }
    if (ws.cell_path) {
        P.add(&ws.grid, 1);
        P.add(&ws.cell_of_atom, n);
        P.add(&ws.cell_rank, n);
        P.add(&ws.cell_count, (size_t)ws.max_cells);
        P.add(&ws.cell_start, (size_t)ws.max_cells + 1);
        P.add(&ws.cell_atoms, n);
    }
}
}  // namespace

size_t workspace_bytes(int cap_atoms, int cap_mols, int precision, bool cell_path, int nbr_cap, int max_cells,
                       int nets) {
    Workspace ws;
    ws.nets = nets;
    ws.cap_atoms = cap_atoms;
    ws.cap_mols = cap_mols;
    ws.rows_cap = rows_capacity(cap_atoms);
    ws.precision = precision;
    ws.cell_path = cell_path;
    ws.nbr_cap = nbr_cap;
    ws.max_cells = max_cells;
    Plan P;
    plan_workspace(P, ws);
    return P.total;
}

int workspace_create(Workspace& ws, int cap_atoms, int cap_mols, int precision, bool cell_path, int nbr_cap,
                     int max_cells, int nets) {
    ws = Workspace();
    ws.nets = nets;
    ws.cap_atoms = cap_atoms;
    ws.cap_mols = cap_mols;
    ws.rows_cap = rows_capacity(cap_atoms);
    ws.precision = precision;
    ws.cell_path = cell_path;
    ws.nbr_cap = nbr_cap;
    ws.max_cells = max_cells;
    Plan P;
    plan_workspace(P, ws);
    // one device block for everything, carved in 256-byte aligned pieces
    char* base = static_cast<char*>(dev_alloc(P.total));
    if (!base) return set_error(-2, "device allocation of %zu bytes failed", P.total);
    ws.owned.push_back(base);
    size_t off = 0;
    for (auto& it : P.items) {
        *it.dst = base + off;
        off += it.bytes;
    }
    ws.bytes = P.total;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&ws.h_ctr), sizeof(Counters));
    if (e != cudaSuccess) {
        workspace_destroy(ws);
        return cuda_error(e, "cudaMallocHost(counters)");
    }
    std::memset(ws.h_ctr, 0, sizeof(Counters));
    // zero-fill: AEV pad columns and rows start at zero
    e = cudaMemset(base, 0, P.total);
    if (e != cudaSuccess) {
        workspace_destroy(ws);
        return cuda_error(e, "cudaMemset(workspace)");
    }
    return 0;
}

void workspace_destroy(Workspace& ws) {
    for (void* p : ws.owned) dev_free(p);
    ws.owned.clear();
    if (ws.h_ctr) cudaFreeHost(ws.h_ctr);
    ws.h_ctr = nullptr;
}

int enqueue_eval(Workspace& ws, const DevWeights& w, const EvalSpec& sp, cudaStream_t st) {
    const int n = sp.n_atoms;
    if (n <= 0 || n > ws.cap_atoms) return set_error(-1, "atom count %d outside [1, %d]", n, ws.cap_atoms);
    if (sp.n_mols > ws.cap_mols) return set_error(-1, "molecule count %d above %d", sp.n_mols, ws.cap_mols);
    const bool batch = sp.d_mol_start != nullptr;
    const bool fast = ws.precision != 0;
    cudaError_t ce;

    AevArgs aa;
    aa.n = n;
    aa.hi = ws.hi;
    aa.lo = ws.lo;
    aa.nbr = ws.nbr;
    aa.nbr_cnt = ws.nbr_cnt;
    aa.cap = ws.nbr_cap;
    aa.box = make_box(batch ? 0 : sp.periodic, sp.L);
    aa.ctr = ws.ctr;
    aa.rank = ws.rank;
    aa.big_list = ws.ang_big_list;
    aa.big_flag = ws.ang_big_flag;

    if (!sp.reuse_aev) {
        ce = cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), st);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaMemsetAsync(counters)");
        if (sp.d_index)
            launch_gather_subset(st, n, sp.d_index, sp.d_coords_full, sp.n_full, const_cast<double*>(sp.d_xyz),
                                 ws.ctr);
        NbrArgs na{ws.hi, ws.lo, ws.nbr, ws.nbr_cnt, ws.nbr_cap, sp.r_list * sp.r_list};
        // a small open system without a persistent list: all pairs of one
        // molecule (2 launches) instead of the cell list (7 launches; launch
        // latency dominates at this size, e.g. a ligand's integrator step)
        const bool small_open = !batch && !sp.periodic && sp.half_skin2 <= 0.f && n <= kAllPairsMaxAtoms;
        if (batch || small_open) {
            launch_stage_batch(st, batch ? sp.n_mols : 1, n, batch ? sp.d_mol_start : nullptr, sp.d_xyz,
                               sp.d_species, ws.hi, ws.lo, ws.rank, ws.ctr, ws.grad);
            launch_nbr_allpairs(st, n, batch ? sp.n_mols : 1, batch ? sp.d_mol_start : nullptr, na, ws.ctr);
        } else {
            if (!ws.cell_path) return set_error(-1, "workspace has no cell list");
            launch_stage_system(st, n, sp.d_xyz, sp.d_species, sp.L, sp.periodic, sp.periodic ? 0 : 1, ws.hi, ws.lo,
                                ws.rank, ws.ctr, ws.grad, ws.ref, sp.half_skin2, sp.force_rebuild ? 1 : 0);
            if (!sp.periodic) launch_grid_setup(st, ws.ctr, ws.grid, sp.r_list, ws.max_cells);
            ce = cudaMemsetAsync(ws.cell_count, 0, sizeof(int) * (size_t)ws.max_cells, st);
            if (ce != cudaSuccess) return cuda_error(ce, "cudaMemsetAsync(cells)");
            launch_cell_build(st, n, ws.hi, ws.grid, ws.max_cells, ws.cell_of_atom, ws.cell_rank, ws.cell_count,
                              ws.cell_start, ws.cell_atoms, ws.ctr);
            launch_nbr_cell(st, n, na, aa.box, ws.grid, ws.cell_of_atom, ws.cell_start, ws.cell_atoms, ws.ctr,
                            ws.ref);
        }
        if (ws.precision == 0)
            launch_aev_f32(st, aa, ws.G32, ws.row_atom, fast);
        else
            launch_aev_bf16(st, aa, ws.G16, ws.G16lo, ws.row_atom, fast);
    }

    if (w.n_nets != ws.nets)
        return set_error(-1, "weights hold %d nets, the workspace was sized for %d", w.n_nets, ws.nets);
    if (ws.precision == 0) {
        // ensemble: one pass per net, each adding its share of the mean
        for (int k = 0; k < w.n_nets; ++k)
            launch_mlp_f32(st, ws.rows_cap, ws.ctr, w.f32[k], ws.G32, ws.row_atom, ws.fb, ws.e, ws.dG,
                           sp.network_backward, k, w.n_nets);
    } else {
        if (!mlp_tc_available()) return set_error(-1, "BF16 tensor-core network is not available in this build");
        if (!launch_mlp_bf16(st, ws.rows_cap, ws.ctr, w.bf16, ws.G16, ws.G16lo, ws.precision == 1, ws.row_atom,
                             ws.e, ws.cap_atoms, ws.dG16, ws.g1ens, sp.network_backward, &ws.ctr->net_error))
            return -5;
    }
    if (sp.network_backward) launch_forces(st, aa, ws.dG, ws.dG16, ws.grad, fast);
    launch_finalize(st, sp.n_mols, sp.d_mol_start, n, ws.e, ws.grad, sp.energy ? sp.d_E : nullptr,
                    sp.network_backward ? sp.d_F : nullptr, sp.d_grad_scale, sp.sign, ws.ctr, ws.err_sticky,
                    sp.d_index, sp.n_full, sp.accumulate, ws.e_nets(), ws.cap_atoms);
    ce = cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return cuda_error(ce, "cudaMemcpyAsync(counters)");
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_error(ce, "kernel launch");
    return 0;
}

int check_counters(const Workspace& ws) {
    const Counters& c = *ws.h_ctr;
    if (c.bad_species & 1) return set_error(-1, "element code outside [0, 7) in the input");
    if (c.bad_species & 2) return set_error(-1, "molecule offsets do not partition [0, n_atoms)");
    if (c.bad_species & 4) return set_error(-1, "ML-region index outside [0, n_full)");
    if (c.nbr_overflow)
        return set_error(-7, "neighbor list overflow: an atom has %d neighbors (capacity %d)", c.nbr_overflow,
                         ws.nbr_cap);
    if (c.ang_overflow)
        return set_error(-7, "too many neighbors inside the angular cutoff (%d; limit %d)", c.ang_overflow,
                         kAngCapBig);
    if (c.net_error)
        return set_error(-5, "tensor-core network kernel gave up on a bounded wait (code %#x)", c.net_error);
    return 0;
}

}  // namespace mlp

// Plan construction and the C ABI entry points (include/st.h, st_stages.h).
//
// A plan holds, on the device and for its whole life, everything that does
// not change between time steps: Gaussian nodes, Legendre tables in the
// layout of the chosen precision, per-row FFT data and the workspace.  This is
// the "reusable arrays" restructuring of ESCAPE D3.3 section 4.2.3 (all
// allocation and set-up hoisted out of the time-step loop) and the flat,
// read-only plan metadata of section 4.2.6.4.
#include "st_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>

namespace st {

static thread_local std::string g_last_error;

void set_last_error(const std::string &s) { g_last_error = s; }

st_status cuda_fail(cudaError_t e, const char *what)
{
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA;
}



static int row_trunc(int T, int n) { return std::min(T, (n - 1) / 2); }

// Factor N into Stockham radices: 4s, then 2, 3, 5, then any other primes.
static int factorize(int N, int *rad)
{
    int n = 0;
    while (N % 4 == 0 && n < MAX_RADICES) { rad[n++] = 4; N /= 4; }
    while (N % 2 == 0 && n < MAX_RADICES) { rad[n++] = 2; N /= 2; }
    while (N % 3 == 0 && n < MAX_RADICES) { rad[n++] = 3; N /= 3; }
    while (N % 5 == 0 && n < MAX_RADICES) { rad[n++] = 5; N /= 5; }
    for (int p = 7; (long long)p * p <= N && n < MAX_RADICES; p += 2)
        while (N % p == 0 && n < MAX_RADICES) { rad[n++] = p; N /= p; }
    if (N > 1 && n < MAX_RADICES) rad[n++] = N;
    return n;
}

// Smallest 2^a 3^b 5^c >= n with a >= 2 (so that radix-4 passes lead).
static int smooth_at_least(int n)
{
    for (int L = std::max(n, 4);; ++L) {
        if (L % 4) continue;
        int q = L;
        while (q % 2 == 0) q /= 2;
        while (q % 3 == 0) q /= 3;
        while (q % 5 == 0) q /= 5;
        if (q == 1) return L;
    }
}

// Order radices so that consecutive pairs (fused into one pass) match a
// large radix with a small one: descending, then largest/smallest alternating.
static void pair_radices(int *rad, int n)
{
    std::vector<int> v(rad, rad + n);
    std::sort(v.begin(), v.end(), [](int a, int b) { return a > b; });
    int lo = 0, hi = n - 1, k = 0;
    while (lo <= hi) {
        rad[k++] = v[lo++];
        if (lo <= hi) rad[k++] = v[hi--];
    }
}

// Stages fused into one pass when the pair has at most this many points
// (must match the FFT kernels).
constexpr int FFT_MAX_FUSED = 16;

// Shared-memory wavefronts of the row's in-place passes under address map
// `mode`, relative to the conflict-free count (8-byte accesses: two phases of
// 16 threads; a phase costs its largest number of distinct addresses that
// share a 8-byte bank slot).  Used to pick the map per row.
static double fft_conflicts(int L, const int *rad, int n, int mode)
{
    struct Pass { int Ns, Ra, Rb; };
    std::vector<Pass> ps;
    int Ns = L;
    for (int q = 0; q < n;) {
        if (q + 1 < n && rad[q] * rad[q + 1] <= FFT_MAX_FUSED) {
            ps.push_back({Ns, rad[q], rad[q + 1]});
            Ns /= rad[q] * rad[q + 1];
            q += 2;
        } else {
            ps.push_back({Ns, rad[q], 1});
            Ns /= rad[q];
            q += 1;
        }
    }
    double tot = 0, ideal = 0;
    for (const Pass &P : ps) {
        const int ma = P.Ns / P.Ra, mb = P.Rb > 1 ? ma / P.Rb : ma, per = L / (P.Ra * P.Rb);
        for (int w0 = 0; w0 < per; w0 += 32) {
            const int nt = std::min(32, per - w0);
            for (int ra = 0; ra < P.Ra; ++ra)
                for (int rb = 0; rb < P.Rb; ++rb)
                    for (int h = 0; h < nt; h += 16) {
                        int addr[16], cnt[16] = {0};
                        int m = 0;
                        for (int t = w0 + h; t < w0 + std::min(nt, h + 16); ++t) {
                            const int b = t / mb, n1 = t % mb;
                            const int i = b * P.Ns + n1 + ra * ma + (P.Rb > 1 ? rb * mb : 0);
                            const int a = fft_swz(i, mode);
                            bool seen = false;
                            for (int u = 0; u < m; ++u) seen |= addr[u] == a;
                            if (!seen) addr[m++] = a;
                        }
                        int worst = 0;
                        for (int u = 0; u < m; ++u) worst = std::max(worst, ++cnt[addr[u] & 15]);
                        tot += worst;
                        ideal += 1;
                    }
        }
    }
    return ideal > 0 ? tot / ideal : 1.0;
}

static int pick_swizzle(int L, const int *rad, int n)
{
    int best = 0;
    double bc = fft_conflicts(L, rad, n, 0);
    for (int mode = 1; mode <= 3; ++mode) {
        double c = fft_conflicts(L, rad, n, mode);
        if (c < bc - 1e-9) { bc = c; best = mode; }
    }
    return best;
}

static bool smooth5(const int *rad, int n)
{
    for (int q = 0; q < n; ++q)
        if (rad[q] > 5) return false;
    return true;
}

template <typename T>
static st_status dmalloc(st_plan *p, T **ptr, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    p->device_bytes += bytes;
    return ST_OK;
}

st_status plan_alloc(st_plan *p, void **ptr, size_t bytes) { return dmalloc(p, ptr, bytes); }

// Owner of a plan's read-only device arrays (shared between plans).
struct TableCore {
    std::vector<void *> ptrs;
    ~TableCore()
    {
        for (void *q : ptrs)
            if (q) cudaFree(q);
    }
};

static void plan_free(st_plan *p)
{
    if (!p) return;
    void *ws[] = {p->fb, p->fbop, p->sop, p->sout, p->err, p->fb2, p->sout2};
    for (void *q : ws)
        if (q) cudaFree(q);
    // derivative table sets are the plan's own
    for (int set = SET_SYN_H; set < NSETS; ++set) {
        if (p->tab[set]) cudaFree(p->tab[set]);
        if (p->groups[set]) cudaFree(p->groups[set]);
    }
    if (!p->core) {
        // creation failed before the read-only arrays were handed to a core
        void *ro[] = {p->mu, p->w, p->rowpairs, p->tw, p->chirp, p->kern, p->tab[0], p->tab[1], p->groups[0],
                      p->groups[1], p->tiles[0], p->tiles[1], p->srow};
        for (void *q : ro)
            if (q) cudaFree(q);
    }
    p->core.reset();
    for (auto &e : p->pending) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    delete p;
}

// Widest table column tile of the direct GEMMs: 160 is the widest at which
// three pipeline stages (2 x 128 x 128 B of data operand + 2 x 160 x 128 B of
// table a stage) fit in shared memory; with 256 (two stages) the direct GEMMs
// ran 9 % slower at T639 O640 x 548 and 7 % at T1279 O1280 x 137, with 128
// (more tiles, the data operand re-read) 3 % slower.
constexpr int TC_NT_DIR = 160;

// Group layout for one direction and precision (see LegGroup).
static void build_groups(st_plan *p, int dir)
{
    const int T = p->T, J = p->J;
    const bool tc = prec_is_tc(p->prec);
    const int kc = tc ? tc_kc(p->prec) : 1;
    // inverse column tile: the table columns are the J northern rows; width
    // from the autotuner if it chose one, else the fewest tiles of <= 256
    int nct_inv = (J + 255) / 256;
    int nt_inv = ((J + nct_inv - 1) / nct_inv + 15) / 16 * 16;
    if (p->nt_inv > 0) {
        nt_inv = std::min(p->nt_inv, (J + 15) / 16 * 16);
        nct_inv = (J + nt_inv - 1) / nt_inv;
    }
    // wavenumbers of the upper half (shorter reductions) may take their own width
    const int m_split = (p->max_m + 1) / 2;
    int nt_hi = nt_inv, nct_hi = nct_inv;
    if (p->nt_inv_hi > 0) {
        nt_hi = std::min(p->nt_inv_hi, (J + 15) / 16 * 16);
        nct_hi = (J + nt_hi - 1) / nt_hi;
    }

    std::vector<LegGroup> &G = p->groups_h[dir];
    G.assign(2 * (T + 1), LegGroup{});
    long long off = 0;
    for (int m = 0; m <= T; ++m) {
        const int Ke = (T - m) / 2 + 1, Ko = (T - m + 1) / 2;
        for (int par = 0; par < 2; ++par) {
            LegGroup g{};
            g.m = m;
            g.p = par;
            const int Km = par ? Ko : Ke;
            const long long srow = p->srow_h[2 * m + par];
            const long long frow = fb_row(p, par, m, 0);
            const bool live = Km > 0 && m <= p->max_m;
            if (dir == 0) {
                g.ncol = J;
                g.K = Km;
                g.r0 = 0;
                g.data_row0 = srow;
                g.out_row0 = frow;
            } else {
                g.ncol = Km;
                g.K = J;
                g.r0 = live ? p->j0[m] : 0;
                g.data_row0 = frow;
                g.out_row0 = srow;
            }
            if (!live) {
                g.ncol = 0;
                g.K = 0;
            }
            if (tc) {
                if (dir == 0) {
                    g.nt = m < m_split ? nt_inv : nt_hi;
                    g.nct = m < m_split ? nct_inv : nct_hi;
                } else {
                    // direct column tiles: the table columns are the K_m
                    // degrees of (m, parity), the fewest tiles of <= TC_NT_DIR
                    int n = std::max(g.ncol, 1);
                    g.nct = (n + TC_NT_DIR - 1) / TC_NT_DIR;
                    g.nt = ((n + g.nct - 1) / g.nct + 15) / 16 * 16;
                }
                g.nkc = (std::max(g.K, 1) + kc - 1) / kc;
                g.tab_off = off;
                if (live) off += (long long)g.nct * g.nkc * 2 * g.nt * 128;
            } else {
                g.nt = SIMT_TILE;
                g.nct = (std::max(g.ncol, 1) + SIMT_TILE - 1) / SIMT_TILE;
                g.nkc = 0;
                g.tab_off = off;
                if (live) off += (long long)g.ncol * g.K;
            }
            G[2 * m + par] = g;
        }
    }
    const size_t el = tc ? 1 : (p->prec == P_FP64 ? 8 : 4);
    p->tab_bytes[dir] = (size_t)off * el;
}

// Groups of a derivative table set: the geometry (and so the table layout)
// of its direction's base set, with the Fourier-buffer halves exchanged on
// the H sets (H_n^m has the opposite parity in mu to Pbar_n^m).
void build_groups_deriv(st_plan *p, int set)
{
    const int base = set_dir(set);
    p->groups_h[set] = p->groups_h[base];
    if (set == SET_SYN_H)
        for (auto &g : p->groups_h[set]) g.out_row0 = fb_row(p, 1 - g.p, g.m, 0);
    if (set == SET_ANA_H1)
        for (auto &g : p->groups_h[set]) g.data_row0 = fb_row(p, 1 - g.p, g.m, 0);
    p->tab_bytes[set] = p->tab_bytes[base];
}

// Work list (group, column tile), heaviest first.
static std::vector<LegTile> build_tiles(const st_plan *p, int dir)
{
    const bool tc = prec_is_tc(p->prec);
    const int kc = tc ? tc_kc(p->prec) : 16;
    std::vector<std::pair<long long, LegTile>> v;
    const auto &G = p->groups_h[dir];
    for (int gi = 0; gi < (int)G.size(); ++gi) {
        const LegGroup &g = G[gi];
        if (g.ncol <= 0 || g.K <= 0) continue;
        int ct0 = 0;
        if (dir == 0) ct0 = p->j0[g.m] / g.nt;  // rows nearer the pole than j0(m) do not keep m
        const long long chunks = (g.K + kc - 1) / kc - g.r0 / kc;
        for (int ct = ct0; ct < g.nct; ++ct) v.push_back({chunks * g.nt, LegTile{gi, ct}});
    }
    std::stable_sort(v.begin(), v.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<LegTile> out;
    out.reserve(v.size());
    for (auto &e : v) out.push_back(e.second);
    return out;
}

// Per-plan workspace for up to max_fields fields, and the error word.  GEMM
// data operands live in buffers of their own, zeroed once here (see st_plan).
static st_status alloc_workspace(st_plan *p, cudaStream_t s)
{
    st_status r;
    if ((r = dmalloc(p, &p->err, sizeof(int)))) return r;
    ST_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), s));
    const int Cp = cols_padded(p->max_fields);
    const int sb = store_bytes(store_of(p->prec)) * store_planes(store_of(p->prec));
    const int ob = p->prec == P_FP64 ? 8 : 4;
    p->fb_bytes = (size_t)fb_rows(p) * Cp * ob;
    p->fbop_bytes = (size_t)fb_rows(p) * Cp * sb;
    p->sop_bytes = (size_t)p->srow_total * Cp * sb;
    p->sout_bytes = (size_t)p->srow_total * Cp * ob;
    if ((r = dmalloc(p, &p->fb, p->fb_bytes))) return r;
    if ((r = dmalloc(p, &p->fbop, p->fbop_bytes))) return r;
    if ((r = dmalloc(p, &p->sop, p->sop_bytes))) return r;
    if ((r = dmalloc(p, &p->sout, p->sout_bytes))) return r;
    ST_CUDA(cudaMemsetAsync(p->fb, 0, p->fb_bytes, s));
    ST_CUDA(cudaMemsetAsync(p->fbop, 0, p->fbop_bytes, s));
    ST_CUDA(cudaMemsetAsync(p->sop, 0, p->sop_bytes, s));
    ST_CUDA(cudaMemsetAsync(p->sout, 0, p->sout_bytes, s));
    p->workspace_bytes = p->fb_bytes + p->fbop_bytes + p->sop_bytes + p->sout_bytes;
    return ST_OK;
}

// Rebuild the Legendre groups, work lists and tables of both directions with
// the plan's current tile choices (used by the autotuner).  The plan must not
// share its tables with another plan.
st_status rebuild_legendre(st_plan *p, cudaStream_t s)
{
    TableCore *core = (TableCore *)p->core.get();
    if (!core || p->core.use_count() != 1) return ST_ERR_BUSY;
    ST_CUDA(cudaStreamSynchronize(s));
    for (int dir = 0; dir < 2; ++dir) {
        void *old[3] = {p->tab[dir], p->groups[dir], p->tiles[dir]};
        for (void *q : old) {
            if (!q) continue;
            cudaFree(q);
            for (auto &c : core->ptrs)
                if (c == q) c = nullptr;
        }
        p->tab[dir] = nullptr;
        p->groups[dir] = nullptr;
        p->tiles[dir] = nullptr;
    }
    p->table_bytes = 0;
    st_status r;
    for (int dir = 0; dir < 2; ++dir) {
        build_groups(p, dir);
        std::vector<LegTile> tl = build_tiles(p, dir);
        p->ntiles[dir] = (int)tl.size();
        if ((r = dmalloc(p, &p->groups[dir], sizeof(LegGroup) * p->groups_h[dir].size()))) return r;
        ST_CUDA(cudaMemcpy(p->groups[dir], p->groups_h[dir].data(), sizeof(LegGroup) * p->groups_h[dir].size(),
                           cudaMemcpyHostToDevice));
        if ((r = dmalloc(p, &p->tiles[dir], sizeof(LegTile) * std::max<size_t>(tl.size(), 1)))) return r;
        if (!tl.empty())
            ST_CUDA(cudaMemcpy(p->tiles[dir], tl.data(), sizeof(LegTile) * tl.size(), cudaMemcpyHostToDevice));
        if ((r = dmalloc(p, &p->tab[dir], p->tab_bytes[dir]))) return r;
        ST_CUDA(cudaMemsetAsync(p->tab[dir], 0, std::max<size_t>(p->tab_bytes[dir], 16), s));
        p->table_bytes += p->tab_bytes[dir];
        core->ptrs.push_back(p->tab[dir]);
        core->ptrs.push_back(p->groups[dir]);
        core->ptrs.push_back(p->tiles[dir]);
    }
    if ((r = launch_tables(p, s))) return r;
    if (p->deriv) {
        for (int set = SET_SYN_H; set < NSETS; ++set) {
            build_groups_deriv(p, set);
            ST_CUDA(cudaMemcpy(p->groups[set], p->groups_h[set].data(), sizeof(LegGroup) * p->groups_h[set].size(),
                               cudaMemcpyHostToDevice));
            if (p->tab[set]) cudaFree(p->tab[set]);
            p->tab[set] = nullptr;
            if ((r = dmalloc(p, &p->tab[set], p->tab_bytes[set]))) return r;
            ST_CUDA(cudaMemsetAsync(p->tab[set], 0, std::max<size_t>(p->tab_bytes[set], 16), s));
        }
        if ((r = launch_tables_deriv(p, s))) return r;
    }
    ST_CUDA(cudaStreamSynchronize(s));
    return ST_OK;
}

std::string tune_key(const st_plan *p, int nfields)
{
    int b = 1;
    while (b < nfields) b <<= 1;
    return std::to_string(p->T) + " " + std::to_string(p->nlat) + " " + std::to_string(p->kind) + " " +
           std::to_string(p->nlon) + " " + std::to_string(p->prec) + " " + std::to_string(b) + " " +
           std::to_string(p->sm_count);
}

// Apply a cached autotuner choice (file named by ST_TUNE_CACHE) for this
// plan's key, if there is one.
static void apply_tune_cache(st_plan *p)
{
    const char *path = getenv("ST_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string key = tune_key(p, p->max_fields);
    char line[512];
    while (fgets(line, sizeof line, f)) {
        std::string l(line);
        if (l.compare(0, key.size() + 1, key + " ") != 0) continue;
        int v0, k0, v1, k1, nt, nth = 0;
        if (sscanf(l.c_str() + key.size() + 1, "| %d %d %d %d %d %d", &v0, &k0, &v1, &k1, &nt, &nth) >= 5) {
            p->fft_var[0] = v0;
            p->fft_kb[0] = k0;
            p->fft_var[1] = v1;
            p->fft_kb[1] = k1;
            p->nt_inv = nt;
            p->nt_inv_hi = nth;
        }
    }
    fclose(f);
}

static st_status plan_build(st_plan *p, cudaStream_t s)
{
    const int T = p->T, nlat = p->nlat, J = nlat / 2;
    p->J = J;
    p->Jp = (int)rows_padded(J);
    apply_tune_cache(p);
    p->rows.resize(nlat);
    for (int j = 0; j < nlat; ++j) {
        if (p->kind == ST_GRID_REGULAR) p->rows[j] = p->nlon;
        else p->rows[j] = 20 + 4 * (std::min(j, nlat - 1 - j) + 1);
    }
    p->npts = 0;
    for (int n : p->rows) p->npts += n;
    p->nspec = (long long)(T + 1) * (T + 2) / 2;
    p->Mrow.resize(J);
    p->max_m = -1;
    for (int j = 0; j < J; ++j) {
        p->Mrow[j] = row_trunc(T, p->rows[j]);
        p->max_m = std::max(p->max_m, p->Mrow[j]);
    }
    if (p->max_m < 0) return ST_ERR_ARG;
    // packed spectral operand: the even then the odd half of every m; group
    // starts 4-aligned for split TF32 (TMA row coordinate), compact otherwise
    p->srow_h.assign(2 * (T + 1), 0);
    {
        long long r = 0;
        for (int m = 0; m <= T; ++m)
            for (int par = 0; par < 2; ++par) {
                if (p->prec == P_TF32X3) r = rows_padded(r);
                p->srow_h[2 * m + par] = r;
                r += par ? (T - m + 1) / 2 : (T - m) / 2 + 1;
            }
        p->srow_total = rows_padded(r);
    }
    p->j0.assign(T + 1, J);
    for (int m = 0; m <= T; ++m)
        for (int j = 0; j < J; ++j)
            if (p->Mrow[j] >= m) { p->j0[m] = j; break; }

    st_status r;

    // nodes and weights
    if ((r = dmalloc(p, &p->mu, sizeof(double) * nlat))) return r;
    if ((r = dmalloc(p, &p->w, sizeof(double) * nlat))) return r;
    if ((r = launch_gauss(nlat, p->mu, p->w, s))) return r;

    // FFT rows: mixed radix over N where N is 5-smooth, otherwise Bluestein
    // over a 5-smooth L >= N + 2M
    p->rowpairs_h.resize(J);
    long long off = 0, tw = 0, nch = 0, nkn = 0;
    std::vector<long long> roff(nlat);
    for (int j = 0; j < nlat; ++j) { roff[j] = off; off += p->rows[j]; }
    p->max_row = p->max_fft = p->max_chirp = p->max_fft_smem = 0;
    for (int j = 0; j < J; ++j) {
        RowPair &rp = p->rowpairs_h[j];
        memset(&rp, 0, sizeof(rp));
        rp.j = j;
        rp.N = p->rows[j];
        rp.M = p->Mrow[j];
        int radN[MAX_RADICES];
        int nN = factorize(rp.N, radN);
        long long prod = 1;
        for (int q = 0; q < nN; ++q) prod *= radN[q];
        if (prod != rp.N) return ST_ERR_UNSUPPORTED;
        // Bluestein length: the circular convolution must hold N + 2M
        // consecutive chirp offsets (inputs at 2M + 1 wavenumbers and N
        // outputs, or the reverse), so L >= N + 2M
        const int L = smooth_at_least(rp.N + 2 * rp.M);
        int radL[MAX_RADICES];
        int nL = factorize(L, radL);
        pair_radices(radN, nN);
        pair_radices(radL, nL);
        rp.fast = -1;
        // FP32 plans: a compile-time plan of length N, else Bluestein on the
        // shortest compile-time plan of length >= N + 2M; the generic kernel
        // only for what neither covers (and for FP64)
        int fid = -1, fL = 0;
        bool fblue = false;
        if (p->prec != P_FP64) {
            for (int id = 0; id < FF_NPLANS && fid < 0; ++id)
                if (ff_length(id) == rp.N) fid = id;
            if (fid < 0) {
                for (int id = 0; id < FF_NPLANS; ++id) {
                    const int Lf = ff_length(id);
                    if (Lf >= rp.N + 2 * rp.M && (fid < 0 || Lf < fL)) { fid = id; fL = Lf; }
                }
                fblue = fid >= 0;
            }
            if (fid >= 0) fL = ff_length(fid);
        }
        if (fid >= 0) {
            rp.fast = fid;
            rp.mode = fblue ? 1 : 0;
            rp.fftlen = fL;
            rp.nrad = ff_radices(fid, rp.rad);
            rp.swz = 0;
            if (fblue) {
                rp.chirp_off = nch;
                rp.kern_off = nkn;
                nch += rp.N;
                nkn += fL;
                p->max_chirp = std::max(p->max_chirp, rp.N);
            }
        } else if (!smooth5(radN, nN)) {
            rp.mode = 1;
            rp.fftlen = L;
            rp.nrad = nL;
            memcpy(rp.rad, radL, sizeof(int) * nL);
            rp.chirp_off = nch;
            rp.kern_off = nkn;
            nch += rp.N;
            nkn += L;
            p->max_chirp = std::max(p->max_chirp, rp.N);
        } else {
            rp.mode = 0;
            rp.fftlen = rp.N;
            rp.nrad = nN;
            memcpy(rp.rad, radN, sizeof(int) * nN);
        }
        if (rp.fast < 0) rp.swz = pick_swizzle(rp.fftlen, rp.rad, rp.nrad);
        p->max_fft_smem = std::max(p->max_fft_smem, fft_swz_size(rp.fftlen, rp.swz));
        rp.tw_off = tw;
        tw += rp.fftlen;
        rp.off_n = roff[j];
        rp.off_s = roff[nlat - 1 - j];
        p->max_row = std::max(p->max_row, rp.N);
        p->max_fft = std::max(p->max_fft, rp.fftlen);
    }
    p->ntw = tw;
    p->nchirp = nch;
    p->nkern = nkn;
    if ((r = dmalloc(p, &p->srow, sizeof(long long) * p->srow_h.size()))) return r;
    ST_CUDA(cudaMemcpyAsync(p->srow, p->srow_h.data(), sizeof(long long) * p->srow_h.size(), cudaMemcpyHostToDevice,
                            s));
    // device copy ordered by padded FFT length, longest first (the FFT
    // launches take rows with equal fields-per-CTA as consecutive runs)
    p->row_order.resize(J);
    for (int j = 0; j < J; ++j) p->row_order[j] = j;
    // (fast rows first, by plan length, longest first)
    std::stable_sort(p->row_order.begin(), p->row_order.end(), [&](int a, int b) {
        const RowPair &x = p->rowpairs_h[a], &y = p->rowpairs_h[b];
        const bool fx = x.fast >= 0, fy = y.fast >= 0;
        if (fx != fy) return fx;
        if (fx) return x.fftlen > y.fftlen;
        return fft_swz_size(x.fftlen, x.swz) > fft_swz_size(y.fftlen, y.swz);
    });
    p->nfast = 0;
    for (int j = 0; j < J; ++j) p->nfast += p->rowpairs_h[j].fast >= 0;
    std::vector<RowPair> sorted(J);
    for (int q = 0; q < J; ++q) sorted[q] = p->rowpairs_h[p->row_order[q]];
    if ((r = dmalloc(p, &p->rowpairs, sizeof(RowPair) * J))) return r;
    ST_CUDA(cudaMemcpyAsync(p->rowpairs, sorted.data(), sizeof(RowPair) * J, cudaMemcpyHostToDevice, s));
    const size_t cs = p->prec == P_FP64 ? 16 : 8;
    if ((r = dmalloc(p, &p->tw, cs * (size_t)tw))) return r;
    if ((r = launch_twiddles(p, s))) return r;
    if (nch > 0) {
        if ((r = dmalloc(p, &p->chirp, cs * (size_t)nch))) return r;
        if ((r = dmalloc(p, &p->kern, cs * 2 * (size_t)nkn))) return r;  // direct, then inverse
        if ((r = launch_bluestein_setup(p, s))) return r;
    }

    // Legendre groups, tiles, tables
    for (int dir = 0; dir < 2; ++dir) {
        build_groups(p, dir);
        std::vector<LegTile> tl = build_tiles(p, dir);
        p->ntiles[dir] = (int)tl.size();
        if ((r = dmalloc(p, &p->groups[dir], sizeof(LegGroup) * p->groups_h[dir].size()))) return r;
        ST_CUDA(cudaMemcpyAsync(p->groups[dir], p->groups_h[dir].data(), sizeof(LegGroup) * p->groups_h[dir].size(),
                                cudaMemcpyHostToDevice, s));
        if ((r = dmalloc(p, &p->tiles[dir], sizeof(LegTile) * std::max<size_t>(tl.size(), 1)))) return r;
        if (!tl.empty())
            ST_CUDA(cudaMemcpyAsync(p->tiles[dir], tl.data(), sizeof(LegTile) * tl.size(), cudaMemcpyHostToDevice, s));
        // the host copy of the tile list must outlive the async copy
        ST_CUDA(cudaStreamSynchronize(s));
        if ((r = dmalloc(p, &p->tab[dir], p->tab_bytes[dir]))) return r;
        ST_CUDA(cudaMemsetAsync(p->tab[dir], 0, std::max<size_t>(p->tab_bytes[dir], 16), s));
        p->table_bytes += p->tab_bytes[dir];
    }
    // tables from the on-disk cache (directory in ST_TABLE_CACHE) when it holds
    // this plan's, else built here and written there
    const char *cache_dir = getenv("ST_TABLE_CACHE");
    bool cached = false;
    if (cache_dir && *cache_dir) {
        ST_CUDA(cudaStreamSynchronize(s));
        cached = load_tables(p, table_cache_path(p, cache_dir).c_str()) == ST_OK;
        set_last_error("");
    }
    if (!cached) {
        if ((r = launch_tables(p, s))) return r;
        p->launches[K_TABLES]++;
        if (cache_dir && *cache_dir) {
            ST_CUDA(cudaStreamSynchronize(s));
            save_tables(p, table_cache_path(p, cache_dir).c_str());  // best effort
            set_last_error("");
        }
    }

    // the read-only arrays now belong to a shareable core
    {
        auto core = std::make_shared<TableCore>();
        core->ptrs = {p->mu, p->w, p->rowpairs, p->tw, p->chirp, p->kern, p->tab[0], p->tab[1], p->groups[0],
                      p->groups[1], p->tiles[0], p->tiles[1], p->srow};
        p->core = core;
    }
    if ((r = alloc_workspace(p, s))) return r;

    if (prec_is_tc(p->prec)) {
        for (int dir = 0; dir < 2; ++dir) {
            int mx = 16;
            for (const auto &g : p->groups_h[dir]) mx = std::max(mx, g.nt);
            int S = 0;
            tc_smem_bytes(p->prec, mx, &S);
            if (S < 2) return ST_ERR_UNSUPPORTED;
        }
    }
    ST_CUDA(cudaStreamSynchronize(s));
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

static st_status check_fields(st_plan_t p, int nfields)
{
    if (!p) return ST_ERR_ARG;
    if (nfields < 1 || nfields > p->max_fields) {
        set_last_error("nfields out of range");
        return ST_ERR_ARG;
    }
    return ST_OK;
}

const char *kernel_name(const st_plan *p, int kind)
{
    const bool tc = prec_is_tc(p->prec);
    switch (kind) {
    case K_PACK: return "pack_spectra";
    case K_LEG_INV: return tc ? "legendre_inverse_tcgen05" : "legendre_inverse_simt";
    case K_FFT_INV: return "fft_inverse";
    case K_FFT_DIR: return "fft_direct";
    case K_LEG_DIR: return tc ? "legendre_direct_tcgen05" : "legendre_direct_simt";
    case K_UNPACK: return "unpack_spectra";
    case K_EXPORT: return "fourier_export";
    case K_TABLES: return "plan_tables";
    case K_COMBINE: return "derivative_combine";
    }
    return "?";
}

static cudaEvent_t take_event(st_plan *p)
{
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int &kernel_launches()
{
    static thread_local int n = 0;
    return n;
}

// Runs one launcher, counting the kernels it launches and, when timing is
// on, bracketing it with events on its stream.
template <class F>
static st_status counted(st_plan *p, int kind, cudaStream_t s, F f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->timing) {
        a = take_event(p);
        b = take_event(p);
        if (a) cudaEventRecord(a, s);
    }
    const int k0 = kernel_launches();
    st_status r = f();
    if (r == ST_OK) p->launches[kind] += kernel_launches() - k0;
    if (p->timing && a && b) {
        cudaEventRecord(b, s);
        p->pending.push_back({kind, a, b});
    } else {
        if (a) p->event_pool.push_back(a);
        if (b) p->event_pool.push_back(b);
    }
    return r;
}

st_status count_launch(st_plan *p, int kind, cudaStream_t s, const std::function<st_status()> &f)
{
    return counted(p, kind, s, f);
}

static st_status leg(st_plan *p, int dir, int nfields, cudaStream_t s)
{
    return counted(p, dir == 0 ? K_LEG_INV : K_LEG_DIR, s, [&] {
        return prec_is_tc(p->prec) ? launch_leg_tc(p, dir, nfields, s) : launch_leg_simt(p, dir, nfields, s);
    });
}
static st_status pack(st_plan *p, const void *spec, int nfields, cudaStream_t s)
{
    return counted(p, K_PACK, s, [&] { return launch_pack(p, spec, nfields, s); });
}
static st_status unpack(st_plan *p, void *spec, int nfields, cudaStream_t s)
{
    return counted(p, K_UNPACK, s, [&] { return launch_unpack(p, spec, nfields, s); });
}
static st_status fft_inv(st_plan *p, void *grid, int nfields, cudaStream_t s)
{
    return counted(p, K_FFT_INV, s, [&] { return launch_fft_inv(p, grid, nfields, s); });
}
static st_status fft_dir(st_plan *p, const void *grid, int nfields, cudaStream_t s)
{
    return counted(p, K_FFT_DIR, s, [&] { return launch_fft_dir(p, grid, nfields, s); });
}

// An empty kernel compiled like every other in the library: its attributes
// tell st_build_info which architecture the library's code targets.
__global__ void k_build_probe() {}

}  // namespace st

using namespace st;

extern "C" {

st_status st_build_info(int *cc_major, int *cc_minor, int *binary_version)
{
    int dev = 0;
    ST_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    ST_CUDA(cudaGetDeviceProperties(&prop, dev));
    cudaFuncAttributes attr;
    ST_CUDA(cudaFuncGetAttributes(&attr, k_build_probe));
    if (cc_major) *cc_major = prop.major;
    if (cc_minor) *cc_minor = prop.minor;
    if (binary_version) *binary_version = attr.binaryVersion;
    return ST_OK;
}

const char *st_status_string(st_status s)
{
    switch (s) {
    case ST_OK: return "ok";
    case ST_ERR_ARG: return "invalid argument";
    case ST_ERR_OOM: return "out of device memory";
    case ST_ERR_CUDA: return "CUDA error";
    case ST_ERR_TIMEOUT: return "device-side wait timed out";
    case ST_ERR_UNSUPPORTED: return "unsupported";
    case ST_ERR_BUSY: return "busy";
    }
    return "unknown status";
}

const char *st_last_error(void) { return g_last_error.c_str(); }

st_status st_plan_create(st_plan_t *out, int T, const st_grid_desc *grid, int prec, int max_fields, void *stream)
{
    if (!out) return ST_ERR_ARG;
    *out = nullptr;
    if (!grid || T < 1 || grid->nlat < 2 || (grid->nlat & 1) || max_fields < 1 || prec < 0 || prec > 3 ||
        (grid->kind != ST_GRID_REGULAR && grid->kind != ST_GRID_OCTAHEDRAL) ||
        (grid->kind == ST_GRID_REGULAR && grid->nlon < 1) || T > 4095 || grid->nlat > 8192 ||
        (grid->kind == ST_GRID_REGULAR && grid->nlon > 65536)) {
        set_last_error("invalid plan arguments");
        return ST_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st_plan *p = new st_plan();
    p->T = T;
    p->nlat = grid->nlat;
    p->kind = grid->kind;
    p->nlon = grid->kind == ST_GRID_REGULAR ? grid->nlon : 0;
    p->prec = prec;
    p->max_fields = max_fields;
    // fast kernels: two CTAs of 256 threads per SM (128 registers a thread);
    // the direct transform in 512-thread CTAs with twice the budget (the
    // autotuner's choice at T639 and T1279)
    if (prec != ST_FP64) {
        p->fft_kb[0] = p->fft_kb[1] = 108;
        p->fft_var[1] = 1;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaGetDevice"); }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, p->device);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaGetDeviceProperties"); }
    p->sm_count = prop.multiProcessorCount;
    if (prec_is_tc(prec) && !(prop.major == 10 && prop.minor == 3)) {
        set_last_error("tensor-core precisions need an sm_103 device");
        plan_free(p);
        return ST_ERR_UNSUPPORTED;
    }
    st_status r = plan_build(p, s);
    if (r != ST_OK) {
        cudaStreamSynchronize(s);
        plan_free(p);
        return r;
    }
    *out = p;
    return ST_OK;
}

st_status st_plan_create_shared(st_plan_t *out, st_plan_t base, int max_fields, void *stream)
{
    if (!out) return ST_ERR_ARG;
    *out = nullptr;
    if (!base || !base->core || max_fields < 1) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    st_plan *p = new st_plan();
    // host metadata and read-only device pointers as in the base plan
    p->T = base->T; p->nlat = base->nlat; p->J = base->J; p->Jp = base->Jp; p->kind = base->kind;
    p->nlon = base->nlon; p->prec = base->prec; p->max_m = base->max_m; p->device = base->device;
    p->sm_count = base->sm_count; p->rows = base->rows; p->Mrow = base->Mrow; p->j0 = base->j0;
    p->npts = base->npts; p->nspec = base->nspec; p->srow_h = base->srow_h; p->srow = base->srow;
    p->srow_total = base->srow_total; p->mu = base->mu; p->w = base->w; p->rowpairs = base->rowpairs;
    p->rowpairs_h = base->rowpairs_h; p->row_order = base->row_order; p->tw = base->tw; p->ntw = base->ntw; p->chirp = base->chirp;
    p->kern = base->kern; p->nchirp = base->nchirp; p->nkern = base->nkern; p->max_row = base->max_row;
    p->max_fft = base->max_fft; p->max_chirp = base->max_chirp; p->max_fft_smem = base->max_fft_smem;
    p->nfast = base->nfast;
    p->fft_var[0] = base->fft_var[0]; p->fft_var[1] = base->fft_var[1];
    p->fft_kb[0] = base->fft_kb[0]; p->fft_kb[1] = base->fft_kb[1]; p->nt_inv = base->nt_inv;
    p->nt_inv_hi = base->nt_inv_hi;
    for (int d = 0; d < 2; ++d) {
        p->tab[d] = base->tab[d];
        p->tab_bytes[d] = base->tab_bytes[d];
        p->groups[d] = base->groups[d];
        p->groups_h[d] = base->groups_h[d];
        p->tiles[d] = base->tiles[d];
        p->ntiles[d] = base->ntiles[d];
    }
    p->table_bytes = base->table_bytes;
    p->core = base->core;
    p->max_fields = max_fields;
    st_status r = alloc_workspace(p, s);
    if (r == ST_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (r != ST_OK) {
        plan_free(p);
        return r;
    }
    *out = p;
    return ST_OK;
}

st_status st_plan_destroy(st_plan_t p)
{
    plan_free(p);
    return ST_OK;
}

st_status st_plan_query(st_plan_t p, st_plan_info *info)
{
    if (!p || !info) return ST_ERR_ARG;
    info->T = p->T;
    info->nlat = p->nlat;
    info->kind = p->kind;
    info->precision = p->prec;
    info->max_fields = p->max_fields;
    info->max_m = p->max_m;
    info->spec_elems = (size_t)p->nspec;
    info->grid_points = (size_t)p->npts;
    info->element_bytes = p->prec == P_FP64 ? 8 : 4;
    info->device_bytes = p->device_bytes;
    info->table_bytes = p->table_bytes;
    info->workspace_bytes = p->workspace_bytes;
    info->launch_shape[0] = p->fft_var[0];
    info->launch_shape[1] = p->fft_kb[0];
    info->launch_shape[2] = p->fft_var[1];
    info->launch_shape[3] = p->fft_kb[1];
    info->launch_shape[4] = p->nt_inv;
    info->launch_shape[5] = p->nt_inv_hi;
    return ST_OK;
}

st_status st_plan_row_lengths(st_plan_t p, int *rows_host)
{
    if (!p || !rows_host) return ST_ERR_ARG;
    memcpy(rows_host, p->rows.data(), sizeof(int) * p->nlat);
    return ST_OK;
}

st_status st_plan_nodes(st_plan_t p, double *mu_host, double *w_host)
{
    if (!p || !mu_host || !w_host) return ST_ERR_ARG;
    ST_CUDA(cudaMemcpy(mu_host, p->mu, sizeof(double) * p->nlat, cudaMemcpyDeviceToHost));
    ST_CUDA(cudaMemcpy(w_host, p->w, sizeof(double) * p->nlat, cudaMemcpyDeviceToHost));
    return ST_OK;
}

st_status st_inv_trans(st_plan_t p, const void *spec_dev, void *grid_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!spec_dev || !grid_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = pack(p, spec_dev, nfields, s))) return r;
    if ((r = leg(p, 0, nfields, s))) return r;
    return fft_inv(p, grid_dev, nfields, s);
}

st_status st_dir_trans(st_plan_t p, const void *grid_dev, void *spec_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!spec_dev || !grid_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = fft_dir(p, grid_dev, nfields, s))) return r;
    if ((r = leg(p, 1, nfields, s))) return r;
    return unpack(p, spec_dev, nfields, s);
}

st_status st_plan_sync(st_plan_t p, void *stream)
{
    if (!p) return ST_ERR_ARG;
    ST_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int e = 0;
    ST_CUDA(cudaMemcpy(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        ST_CUDA(cudaMemset(p->err, 0, sizeof(int)));
        set_last_error("device-side wait timed out (flags " + std::to_string(e) + ")");
        return ST_ERR_TIMEOUT;
    }
    return ST_OK;
}

// ---- stages

st_status st_gauss_nodes(int nlat, double *mu_dev, double *w_dev, void *stream)
{
    if (nlat < 2 || !mu_dev || !w_dev) return ST_ERR_ARG;
    return launch_gauss(nlat, mu_dev, w_dev, (cudaStream_t)stream);
}

st_status st_legendre_values(int T, const double *mu_dev, int nmu, double *out_dev, void *stream)
{
    if (T < 0 || nmu < 1 || !mu_dev || !out_dev) return ST_ERR_ARG;
    return launch_legendre_values(T, mu_dev, nmu, out_dev, (cudaStream_t)stream);
}

st_status st_inv_legendre(st_plan_t p, const void *spec_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!spec_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = pack(p, spec_dev, nfields, s))) return r;
    return leg(p, 0, nfields, s);
}

st_status st_inv_fft(st_plan_t p, void *grid_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!grid_dev) return ST_ERR_ARG;
    return fft_inv(p, grid_dev, nfields, (cudaStream_t)stream);
}

st_status st_dir_fft(st_plan_t p, const void *grid_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!grid_dev) return ST_ERR_ARG;
    return fft_dir(p, grid_dev, nfields, (cudaStream_t)stream);
}

st_status st_dir_legendre(st_plan_t p, void *spec_dev, int nfields, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!spec_dev) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = leg(p, 1, nfields, s))) return r;
    return unpack(p, spec_dev, nfields, s);
}

st_status st_fourier_export(st_plan_t p, int direction, int nfields, double *out_dev, void *stream)
{
    st_status r = check_fields(p, nfields);
    if (r) return r;
    if (!out_dev || direction < 0 || direction > 1) return ST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    return counted(p, K_EXPORT, s, [&] { return launch_fourier_export(p, direction, nfields, out_dev, s); });
}

st_status st_plan_inject(st_plan_t p, int what, unsigned wait_ms)
{
    if (!p || what < 0 || what > 1 || (what == 1 && (wait_ms < 1 || wait_ms > 2000))) return ST_ERR_ARG;
    if (!prec_is_tc(p->prec)) return ST_ERR_UNSUPPORTED;
    p->inject_withhold = what;
    p->inject_wait_ns = (unsigned long long)wait_ms * 1000000ull;
    return ST_OK;
}

st_status st_plan_set_timing(st_plan_t p, int enable)
{
    if (!p) return ST_ERR_ARG;
    p->timing = enable != 0;
    return ST_OK;
}

st_status st_plan_timings(st_plan_t p, st_kernel_time *out, int max, int *n)
{
    if (!p || (!out && max > 0)) return ST_ERR_ARG;
    for (auto &e : p->pending) {
        float ms = 0.f;
        ST_CUDA(cudaEventSynchronize(e.b));
        ST_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
        p->total_ms[e.kind] += ms;
        p->timed[e.kind]++;
        p->event_pool.push_back(e.a);
        p->event_pool.push_back(e.b);
    }
    p->pending.clear();
    int k = 0;
    for (int i = 0; i < K_NKINDS; ++i) {
        if (p->launches[i] == 0) continue;
        if (k < max) {
            out[k].name = kernel_name(p, i);
            out[k].launches = p->launches[i];
            out[k].total_ms = p->total_ms[i];
            out[k].timed = p->timed[i];
        }
        ++k;
    }
    if (n) *n = k;
    return ST_OK;
}

st_status st_plan_reset_timings(st_plan_t p)
{
    if (!p) return ST_ERR_ARG;
    for (auto &e : p->pending) {
        cudaEventSynchronize(e.b);
        p->event_pool.push_back(e.a);
        p->event_pool.push_back(e.b);
    }
    p->pending.clear();
    for (int i = 0; i < 16; ++i) {
        p->launches[i] = 0;
        p->timed[i] = 0;
        p->total_ms[i] = 0;
    }
    return ST_OK;
}

}  // extern "C"

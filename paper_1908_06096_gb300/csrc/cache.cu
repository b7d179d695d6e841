// On-disk cache of a plan's tables (include/st.h: st_plan_save_tables,
// st_plan_load_tables, and the ST_TABLE_CACHE directory st_plan_create
// consults).  The paper's SH dwarf rebuilds nothing per time step (section
// 4.2.3); this keeps the once-per-run work -- Gaussian nodes and weights and
// the Legendre tables in the plan's precision and layout -- across runs, the
// way a model restarts from a checkpoint.
//
// File: a fixed header (magic, format version, the plan facts the tables
// depend on, the payload sizes, an FNV-1a checksum of the payload), then mu,
// w and the two table sets, byte for byte as they sit on the device.
#include "st_internal.cuh"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace st {

namespace {

constexpr char kMagic[8] = {'S', 'T', 'T', 'A', 'B', 'L', 'E', 'S'};
// 2: the direct tables' column tiles are at most 160 columns wide (files of
// format 1 hold the 256-wide layout and are rebuilt)
constexpr uint32_t kVersion = 2;

struct Header {
    char magic[8];
    uint32_t version;
    int32_t T, nlat, kind, nlon, prec, nt_inv, max_m;
    uint64_t bytes[4];  // mu, w, table set 0, table set 1
    uint64_t checksum;
};

uint64_t fnv1a(uint64_t h, const unsigned char *p, size_t n)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

void fill_header(const st_plan *p, Header *h)
{
    memset(h, 0, sizeof(*h));
    memcpy(h->magic, kMagic, 8);
    h->version = kVersion;
    h->T = p->T;
    h->nlat = p->nlat;
    h->kind = p->kind;
    h->nlon = p->nlon;
    h->prec = p->prec;
    h->nt_inv = p->nt_inv;
    h->max_m = p->max_m;
    h->bytes[0] = h->bytes[1] = sizeof(double) * (uint64_t)p->nlat;
    h->bytes[2] = p->tab_bytes[0];
    h->bytes[3] = p->tab_bytes[1];
}

// Device arrays in file order.
void payload(st_plan *p, void *arr[4])
{
    arr[0] = p->mu;
    arr[1] = p->w;
    arr[2] = p->tab[0];
    arr[3] = p->tab[1];
}

constexpr size_t kChunk = 64u << 20;

}  // namespace

std::string table_cache_path(const st_plan *p, const char *dir)
{
    char name[160];
    snprintf(name, sizeof name, "st_tables_T%d_nlat%d_kind%d_nlon%d_prec%d_nt%d_v%u.bin", p->T, p->nlat, p->kind,
             p->nlon, p->prec, p->nt_inv, kVersion);
    std::string d(dir);
    if (!d.empty() && d.back() != '/') d += '/';
    return d + name;
}

st_status save_tables(st_plan *p, const char *path)
{
    Header h;
    fill_header(p, &h);
    void *arr[4];
    payload(p, arr);
    // checksum first (one pass through host memory per chunk), then write
    std::vector<unsigned char> buf(kChunk);
    uint64_t sum = 1469598103934665603ull;
    for (int a = 0; a < 4; ++a)
        for (uint64_t off = 0; off < h.bytes[a]; off += kChunk) {
            const size_t n = (size_t)std::min<uint64_t>(kChunk, h.bytes[a] - off);
            ST_CUDA(cudaMemcpy(buf.data(), (const char *)arr[a] + off, n, cudaMemcpyDeviceToHost));
            sum = fnv1a(sum, buf.data(), n);
        }
    h.checksum = sum;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) {
        set_last_error(std::string("cannot write ") + tmp);
        return ST_ERR_ARG;
    }
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    for (int a = 0; a < 4 && ok; ++a)
        for (uint64_t off = 0; off < h.bytes[a] && ok; off += kChunk) {
            const size_t n = (size_t)std::min<uint64_t>(kChunk, h.bytes[a] - off);
            if (cudaMemcpy(buf.data(), (const char *)arr[a] + off, n, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
            else ok = fwrite(buf.data(), 1, n, f) == n;
        }
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        set_last_error(std::string("writing the table cache ") + path + " failed");
        return ST_ERR_ARG;
    }
    return ST_OK;
}

st_status load_tables(st_plan *p, const char *path)
{
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_last_error(std::string("cannot open ") + path);
        return ST_ERR_ARG;
    }
    Header h, want;
    fill_header(p, &want);
    bool ok = fread(&h, sizeof h, 1, f) == 1 && memcmp(h.magic, kMagic, 8) == 0 && h.version == kVersion &&
              h.T == want.T && h.nlat == want.nlat && h.kind == want.kind && h.nlon == want.nlon &&
              h.prec == want.prec && h.nt_inv == want.nt_inv && h.max_m == want.max_m &&
              memcmp(h.bytes, want.bytes, sizeof h.bytes) == 0;
    if (!ok) {
        fclose(f);
        set_last_error(std::string(path) + " holds tables of another plan or format");
        return ST_ERR_ARG;
    }
    // read everything into host memory and verify before touching the device
    std::vector<std::vector<unsigned char>> data(4);
    uint64_t sum = 1469598103934665603ull;
    for (int a = 0; a < 4 && ok; ++a) {
        data[a].resize(h.bytes[a]);
        ok = fread(data[a].data(), 1, h.bytes[a], f) == h.bytes[a];
        if (ok) sum = fnv1a(sum, data[a].data(), h.bytes[a]);
    }
    fclose(f);
    if (!ok || sum != h.checksum) {
        set_last_error(std::string(path) + " is truncated or damaged (checksum)");
        return ST_ERR_ARG;
    }
    void *arr[4];
    payload(p, arr);
    for (int a = 0; a < 4; ++a)
        if (h.bytes[a]) ST_CUDA(cudaMemcpy(arr[a], data[a].data(), h.bytes[a], cudaMemcpyHostToDevice));
    return ST_OK;
}

}  // namespace st

using namespace st;

extern "C" {

st_status st_plan_save_tables(st_plan_t p, const char *path)
{
    if (!p || !path) return ST_ERR_ARG;
    ST_CUDA(cudaDeviceSynchronize());
    return save_tables(p, path);
}

st_status st_plan_load_tables(st_plan_t p, const char *path)
{
    if (!p || !path) return ST_ERR_ARG;
    if (p->core && p->core.use_count() != 1) {
        set_last_error("the plan shares its tables with another plan");
        return ST_ERR_BUSY;
    }
    ST_CUDA(cudaDeviceSynchronize());
    return load_tables(p, path);
}

}  // extern "C"

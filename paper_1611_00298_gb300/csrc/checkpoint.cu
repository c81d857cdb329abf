// Checkpoint / resume of the HMC state (Sec. 5 production runs restart from
// saved configurations): the gauge field and the momenta in the host
// canonical layout, as a binary file with a header and a checksum.
//
// File: header (64 bytes, little-endian) then the data as FP64.
//   char[8]   magic "EOFACKPT"
//   uint32    version (1)
//   uint32    kind (EOFA_CKPT_GAUGE, EOFA_CKPT_MOMENTA)
//   int32[4]  dims {X, Y, Z, T}
//   uint64    number of doubles that follow (72 V for both kinds)
//   int64     trajectory number (caller's value)
//   uint64    FNV-1a 64 checksum of the data bytes
//   uint64    reserved (0)
#include "api_util.h"

#include <cstdio>
#include <cstring>
#include <vector>

namespace {

const char kMagic[8] = {'E', 'O', 'F', 'A', 'C', 'K', 'P', 'T'};

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t kind;
    int32_t dims[4];
    uint64_t ndoubles;
    int64_t traj;
    uint64_t checksum;
    uint64_t reserved;
};
static_assert(sizeof(Header) == 64, "checkpoint header is 64 bytes");

// FNV-1a, 64 bit (offset basis 0xcbf29ce484222325, prime 0x100000001b3)
uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 0xCBF29CE484222325ULL;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001B3ULL;
    }
    return h;
}

uint64_t expected_doubles(const int dims[4]) {
    return 72ULL * (uint64_t)dims[0] * dims[1] * dims[2] * dims[3];
}

bool dims_ok(const int dims[4]) {
    for (int k = 0; k < 4; k++)
        if (dims[k] < 2 || (dims[k] & 1)) return false;
    return true;
}

}  // namespace

extern "C" {

int eofa_checkpoint_write(const char* path, int kind, const int dims[4], long long traj, const double* data) {
    if (!path || !dims || !data || (kind != EOFA_CKPT_GAUGE && kind != EOFA_CKPT_MOMENTA) || !dims_ok(dims))
        return EOFA_EINVAL;
    Header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.kind = (uint32_t)kind;
    for (int k = 0; k < 4; k++) h.dims[k] = dims[k];
    h.ndoubles = expected_doubles(dims);
    h.traj = traj;
    const size_t nbytes = h.ndoubles * sizeof(double);
    h.checksum = fnv1a((const unsigned char*)data, nbytes);
    FILE* f = std::fopen(path, "wb");
    if (!f) return EOFA_EINVAL;
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(data, 1, nbytes, f) == nbytes;
    const bool closed = std::fclose(f) == 0;
    return ok && closed ? EOFA_OK : EOFA_EDEVICE;
}

int eofa_checkpoint_read(const char* path, int kind, const int dims[4], long long* traj, double* data) {
    if (!path || !dims || !data || (kind != EOFA_CKPT_GAUGE && kind != EOFA_CKPT_MOMENTA) || !dims_ok(dims))
        return EOFA_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return EOFA_EINVAL;
    Header h;
    int rc = EOFA_OK;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 ||
        h.kind != (uint32_t)kind || h.ndoubles != expected_doubles(dims)) {
        rc = EOFA_EINVAL;
    }
    for (int k = 0; k < 4 && rc == EOFA_OK; k++)
        if (h.dims[k] != dims[k]) rc = EOFA_EINVAL;
    if (rc == EOFA_OK) {
        const size_t nbytes = h.ndoubles * sizeof(double);
        std::vector<unsigned char> buf(nbytes);
        char extra;
        if (std::fread(buf.data(), 1, nbytes, f) != nbytes || std::fread(&extra, 1, 1, f) != 0) rc = EOFA_EINVAL;
        else if (fnv1a(buf.data(), nbytes) != h.checksum) rc = EOFA_EINVAL;
        else {
            std::memcpy(data, buf.data(), nbytes);
            if (traj) *traj = h.traj;
        }
    }
    std::fclose(f);
    return rc;
}

int eofa_gauge_save(eofa_ctx* ctx, const char* path, long long traj) {
    if (!ctx || !path) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        require_gauge(ctx);
        const size_t n = (size_t)ctx->V * 4 * 9 * 2;
        std::vector<double> host(n);
        const double* Uc = (const double*)ctx_buffer(ctx, "U", 0);
        EOFA_CUDA(cudaMemcpy(host.data(), Uc, n * sizeof(double), cudaMemcpyDeviceToHost));
        const int rc = eofa_checkpoint_write(path, EOFA_CKPT_GAUGE, ctx->dims, traj, host.data());
        if (rc != EOFA_OK) return fail(ctx, rc, std::string("cannot write checkpoint ") + path);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_gauge_restore(eofa_ctx* ctx, const char* path, long long* traj) {
    if (!ctx || !path) return fail(ctx, EOFA_EINVAL, "null argument");
    std::vector<double> host((size_t)ctx->V * 4 * 9 * 2);
    const int rc = eofa_checkpoint_read(path, EOFA_CKPT_GAUGE, ctx->dims, traj, host.data());
    if (rc != EOFA_OK)
        return fail(ctx, rc, std::string("checkpoint ") + path + " is missing, of another lattice or corrupt");
    return eofa_gauge_load(ctx, host.data());
}

}  // extern "C"

// Checkpoints of single-cavity handles: lbmfvm_save, lbmfvm_load and the
// host-only lbmfvm_checkpoint_info.  Included by lbmfvm.cu (it needs the
// handle's internals).  The file layout is the one include/lbmfvm.h documents:
// a 256-byte header, then both population buffers (the current post-collision
// state and the previous one, from which the fields at the current step are
// read), the temperature and the residual snapshot, all without row padding.

namespace {

static_assert(sizeof(lbmfvm_checkpoint_header_t) == 256, "checkpoint headers are 256 bytes");
static_assert(offsetof(lbmfvm_checkpoint_header_t, header_crc) == 252, "the header CRC closes the header");

constexpr char kCkptMagic[8] = {'L', 'B', 'M', 'F', 'V', 'M', 'C', '1'};
constexpr uint32_t kCkptVersion = 1;

// CRC-32 of the ISO-HDLC polynomial (reflected 0xEDB88320, initial and final
// complement), one byte at a time from a 256-entry table: crc32_update(0, p, n)
// is the standard checksum of n bytes, and feeding a buffer in pieces gives
// the checksum of the whole.
uint32_t crc32_update(uint32_t crc, const void *data, size_t n) {
    static uint32_t table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint32_t i = 0; i < 256; i++) {
            uint32_t c = i;
            for (int k = 0; k < 8; k++) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
    });
    const uint8_t *p = static_cast<const uint8_t *>(data);
    crc = ~crc;
    for (size_t i = 0; i < n; i++) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

// Payload bytes of a checkpoint of an nx x ny grid in storage prec (0 for an
// unknown precision).
uint64_t ckpt_payload_bytes(int nx, int ny, int prec, int energy) {
    const uint64_t n = (uint64_t)nx * (uint64_t)ny;
    const uint64_t ss = store_size(prec), ts = temp_size(prec);
    if (ss == 0 || (energy != LBMFVM_ENERGY_FV && energy != LBMFVM_ENERGY_LBM_D2Q5)) return 0;
    const uint64_t g = energy == LBMFVM_ENERGY_LBM_D2Q5 ? 2 * 5 * n * ss : 0;
    return 2 * 9 * n * ss + n * ts + 2 * n * sizeof(double) + g;
}

struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) std::fclose(f);
    }
};

// Reads and verifies the checkpoint at path; the payload goes to *payload when
// it is not NULL.  On failure returns LBMFVM_ERR_IO with the reason in why.
int read_checkpoint(const char *path, lbmfvm_checkpoint_header_t *hd, std::vector<uint8_t> *payload, char *why,
                    size_t why_len) {
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) {
        snprintf(why, why_len, "cannot open checkpoint %s", path);
        return LBMFVM_ERR_IO;
    }
    if (std::fread(hd, 1, sizeof(*hd), fc.f) != sizeof(*hd)) {
        snprintf(why, why_len, "checkpoint %s is shorter than its header", path);
        return LBMFVM_ERR_IO;
    }
    if (std::memcmp(hd->magic, kCkptMagic, sizeof(kCkptMagic)) != 0 || hd->version != kCkptVersion ||
        hd->header_bytes != sizeof(*hd)) {
        snprintf(why, why_len, "%s is not a version-%u lbmfvm checkpoint", path, kCkptVersion);
        return LBMFVM_ERR_IO;
    }
    if (crc32_update(0, hd, offsetof(lbmfvm_checkpoint_header_t, header_crc)) != hd->header_crc) {
        snprintf(why, why_len, "checkpoint %s: header CRC mismatch", path);
        return LBMFVM_ERR_IO;
    }
    const uint64_t want = ckpt_payload_bytes(hd->nx, hd->ny, hd->store, hd->energy);
    if (hd->nx < 3 || hd->ny < 3 || (int64_t)hd->nx * hd->ny > (int64_t(1) << 30) || want == 0 ||
        hd->payload_bytes != want) {
        snprintf(why, why_len, "checkpoint %s: payload size does not match its %d x %d grid", path, hd->nx, hd->ny);
        return LBMFVM_ERR_IO;
    }
    if (payload) {
        payload->resize(want);
        if (std::fread(payload->data(), 1, want, fc.f) != want) {
            snprintf(why, why_len, "checkpoint %s is truncated", path);
            return LBMFVM_ERR_IO;
        }
        if (crc32_update(0, payload->data(), want) != hd->payload_crc) {
            snprintf(why, why_len, "checkpoint %s: payload CRC mismatch", path);
            return LBMFVM_ERR_IO;
        }
    } else {
        std::vector<uint8_t> buf(1 << 20);
        uint32_t crc = 0;
        uint64_t left = want;
        while (left > 0) {
            const size_t k = left < buf.size() ? (size_t)left : buf.size();
            if (std::fread(buf.data(), 1, k, fc.f) != k) {
                snprintf(why, why_len, "checkpoint %s is truncated", path);
                return LBMFVM_ERR_IO;
            }
            crc = crc32_update(crc, buf.data(), k);
            left -= k;
        }
        if (crc != hd->payload_crc) {
            snprintf(why, why_len, "checkpoint %s: payload CRC mismatch", path);
            return LBMFVM_ERR_IO;
        }
    }
    if (std::fgetc(fc.f) != EOF) {
        snprintf(why, why_len, "checkpoint %s has bytes after its payload", path);
        return LBMFVM_ERR_IO;
    }
    return LBMFVM_OK;
}

}  // namespace

extern "C" {

int lbmfvm_checkpoint_info(const char *path, lbmfvm_checkpoint_header_t *header) {
    if (!path || !header) return fail_thread(LBMFVM_ERR_ARG, "path or header is NULL");
    char why[512];
    if (int r = read_checkpoint(path, header, nullptr, why, sizeof(why))) return fail_thread(r, "%s", why);
    return LBMFVM_OK;
}

int lbmfvm_save(lbmfvm_t *h, const char *path) {
    if (!h || !path) return fail_thread(LBMFVM_ERR_ARG, "handle or path is NULL");
    if (!h->atlas_cavs.empty()) return fail(h, LBMFVM_ERR_ARG, "checkpoints hold single-cavity handles");
    if (h->grid2) return fail(h, LBMFVM_ERR_ARG, "checkpoints hold handles of grid setting 1");
    const int nx = h->grid.nx, ny = h->grid.ny;
    const size_t n = (size_t)nx * ny, ss = store_size(h->prec), ts = temp_size(h->prec);
    std::vector<uint8_t> payload(ckpt_payload_bytes(nx, ny, h->prec, h->energy));
    if (int r = join_in(h)) return r;
    uint8_t *dst = payload.data();
    // f*^n, then f*^(n-1): nine planes of ny rows each, one 2-D copy per buffer
    for (int b = 0; b < 2; b++) {
        const int buf = b == 0 ? h->parity : h->parity ^ 1;
        CU(h, cudaMemcpy2DAsync(dst, nx * ss, h->base + h->L.f[buf], (size_t)h->L.pitch * ss, nx * ss, 9 * (size_t)ny,
                                cudaMemcpyDeviceToHost, h->s));
        dst += 9 * n * ss;
    }
    CU(h, cudaMemcpy2DAsync(dst, nx * ts, h->base + h->L.T[h->parity], (size_t)h->L.pitch * ts, nx * ts, (size_t)ny,
                            cudaMemcpyDeviceToHost, h->s));
    dst += n * ts;
    CU(h, cudaMemcpyAsync(dst, h->base + h->L.snap, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    dst += 2 * n * sizeof(double);
    // energy populations g*^n, then g*^(n-1)
    for (int b = 0; b < 2 && h->energy == LBMFVM_ENERGY_LBM_D2Q5; b++) {
        const int buf = b == 0 ? h->parity : h->parity ^ 1;
        CU(h, cudaMemcpy2DAsync(dst, nx * ss, h->base + h->L.g[buf], (size_t)h->L.pitch * ss, nx * ss, 5 * (size_t)ny,
                                cudaMemcpyDeviceToHost, h->s));
        dst += 5 * n * ss;
    }
    CU(h, cudaStreamSynchronize(h->s));
    if (int r = check_device_status(h)) return r;

    lbmfvm_checkpoint_header_t hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kCkptMagic, sizeof(kCkptMagic));
    hd.version = kCkptVersion;
    hd.header_bytes = sizeof(hd);
    hd.nx = nx;
    hd.ny = ny;
    hd.store = h->prec;
    hd.steps = h->steps;
    for (int s = 0; s < 4; s++) {
        hd.bc[s] = h->grid.bc[s];
        hd.t_wall[s] = h->grid.t_wall[s];
    }
    hd.u_lid = h->grid.u_lid;
    hd.tau = h->tau;
    hd.alpha = h->alpha;
    hd.gbeta = h->gbeta;
    hd.t_ref = h->t_ref;
    hd.force[0] = h->force[0];
    hd.force[1] = h->force[1];
    hd.payload_bytes = payload.size();
    hd.code_crc = h->code_crc;
    hd.fv_scheme = h->fv_quick ? LBMFVM_FV_QUICK : LBMFVM_FV_CENTRAL;
    hd.fv_substeps = h->fv_sub;
    hd.energy = h->energy;
    hd.wall_bc = h->wall_bc;
    hd.payload_crc = crc32_update(0, payload.data(), payload.size());
    hd.header_crc = crc32_update(0, &hd, offsetof(lbmfvm_checkpoint_header_t, header_crc));

    // Written to path.tmp, flushed to the disk, then renamed over path: a
    // save that fails part-way (a full disk, a killed process) leaves the
    // previous checkpoint at path intact.
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(h, LBMFVM_ERR_IO, "cannot open %s for writing", tmp.c_str());
    bool ok = std::fwrite(&hd, 1, sizeof(hd), f) == sizeof(hd) &&
              std::fwrite(payload.data(), 1, payload.size(), f) == payload.size();
    ok = ok && std::fflush(f) == 0 && fsync(fileno(f)) == 0;
    ok = std::fclose(f) == 0 && ok;
    if (ok) ok = std::rename(tmp.c_str(), path) == 0;
    if (!ok) {
        std::remove(tmp.c_str());
        return fail(h, LBMFVM_ERR_IO, "writing checkpoint %s failed (any earlier file there is unchanged)", path);
    }
    return join_out(h);
}

int lbmfvm_load(lbmfvm_t *h, const char *path) {
    if (!h || !path) return fail_thread(LBMFVM_ERR_ARG, "handle or path is NULL");
    if (!h->atlas_cavs.empty()) return fail(h, LBMFVM_ERR_ARG, "checkpoints hold single-cavity handles");
    if (h->grid2) return fail(h, LBMFVM_ERR_ARG, "checkpoints hold handles of grid setting 1");
    lbmfvm_checkpoint_header_t hd;
    std::vector<uint8_t> payload;
    char why[512];
    if (int r = read_checkpoint(path, &hd, &payload, why, sizeof(why))) return fail(h, r, "%s", why);
    // the handle must be the one the state belongs to
    const char *diff = nullptr;
    if (hd.nx != h->grid.nx || hd.ny != h->grid.ny) diff = "grid size";
    else if (hd.store != h->prec) diff = "storage type";
    else if (hd.code_crc != h->code_crc) diff = "node codes (boundaries or obstacle mask)";
    else if (hd.tau != h->tau || hd.alpha != h->alpha || hd.gbeta != h->gbeta || hd.force[0] != h->force[0] ||
             hd.force[1] != h->force[1] || !(hd.t_ref == h->t_ref))
        diff = "lattice parameters";
    else if (hd.u_lid != h->grid.u_lid) diff = "lid velocity";
    else if (hd.fv_scheme != (h->fv_quick ? LBMFVM_FV_QUICK : LBMFVM_FV_CENTRAL) ||
             (hd.fv_substeps < 1 ? 1 : hd.fv_substeps) != h->fv_sub)
        diff = "energy-update scheme or sub-steps";
    else if (hd.energy != h->energy) diff = "energy solver";
    else if (hd.wall_bc != h->wall_bc) diff = "wall treatment";
    for (int s = 0; s < 4 && !diff; s++)
        if (hd.bc[s] != h->grid.bc[s] || hd.t_wall[s] != h->grid.t_wall[s]) diff = "boundary conditions";
    if (diff) return fail(h, LBMFVM_ERR_ARG, "checkpoint %s was saved with other %s", path, diff);

    const int nx = h->grid.nx, ny = h->grid.ny;
    const size_t n = (size_t)nx * ny, ss = store_size(h->prec), ts = temp_size(h->prec);
    if (int r = join_in(h)) return r;
    const uint8_t *src = payload.data();
    // the current state goes to buffer 0, the previous one to buffer 1
    for (int b = 0; b < 2; b++) {
        CU(h, cudaMemcpy2DAsync(h->base + h->L.f[b], (size_t)h->L.pitch * ss, src, nx * ss, nx * ss, 9 * (size_t)ny,
                                cudaMemcpyHostToDevice, h->s));
        src += 9 * n * ss;
    }
    CU(h, cudaMemcpy2DAsync(h->base + h->L.T[0], (size_t)h->L.pitch * ts, src, nx * ts, nx * ts, (size_t)ny,
                            cudaMemcpyHostToDevice, h->s));
    src += n * ts;
    CU(h, cudaMemcpyAsync(h->base + h->L.snap, src, 2 * n * sizeof(double), cudaMemcpyHostToDevice, h->s));
    src += 2 * n * sizeof(double);
    for (int b = 0; b < 2 && h->energy == LBMFVM_ENERGY_LBM_D2Q5; b++) {
        CU(h, cudaMemcpy2DAsync(h->base + h->L.g[b], (size_t)h->L.pitch * ss, src, nx * ss, nx * ss, 5 * (size_t)ny,
                                cudaMemcpyHostToDevice, h->s));
        src += 5 * n * ss;
    }
    if (int r = clear_tile_counters(h)) return r;
    CU(h, cudaStreamSynchronize(h->s));
    h->parity = 0;
    h->steps = hd.steps;
    return join_out(h);
}

}  // extern "C"

// C ABI of libdnnmg (include/dnnmg.h): argument checks, handles, per-mesh
// element constants, and the ordered launch sequence of one correction step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace dnnmg {

namespace {
thread_local std::string g_error;
}

int fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

void clear_error() { g_error.clear(); }

int round_up(int v, int m) { return (v + m - 1) / m * m; }
size_t align256(size_t v) { return (v + 255) / 256 * 256; }

cudaError_t launch_gru_cuda_core(const Net &n, const void *X, void *h, void *d, int P,
                                 cudaStream_t st);

namespace {

constexpr double kPi = 3.14159265358979323846;

// Coarse solid mask by the centroid test (Sec. 6.1 geometry on a structured mesh).
std::vector<uint8_t> solid_mask(const dnnmg_mesh_desc &d) {
    std::vector<uint8_t> m((size_t)d.nxc * d.nyc, 0);
    if (d.solid) {
        for (size_t i = 0; i < m.size(); ++i) m[i] = d.solid[i] ? 1 : 0;
        return m;
    }
    if (!(d.obst_ax > 0 && d.obst_ay > 0)) return m;
    const double hx = d.lx / d.nxc, hy = d.ly / d.nyc;
    for (int j = 0; j < d.nyc; ++j)
        for (int i = 0; i < d.nxc; ++i) {
            const double xc = (i + 0.5) * hx, yc = (j + 0.5) * hy;
            const double tx = (xc - d.obst_cx) / d.obst_ax, ty = (yc - d.obst_cy) / d.obst_ay;
            const double tx2 = tx * tx, ty2 = ty * ty;
            m[(size_t)j * d.nxc + i] = (tx2 + ty2 < 1.0) ? 1 : 0;
        }
    return m;
}

// Fluid patch numbering: lexicographic over the patch grid, patch-x fastest.
int patch_numbering(const dnnmg_mesh_desc &d, const std::vector<uint8_t> &solid,
                    std::vector<int> *id, std::vector<int> *cell) {
    const int npx = d.nxc / d.s, npy = d.nyc / d.s;
    if (id) id->assign((size_t)npx * npy, -1);
    if (cell) cell->clear();
    int P = 0;
    for (int pj = 0; pj < npy; ++pj)
        for (int pi = 0; pi < npx; ++pi) {
            bool fluid = false;
            for (int b = 0; b < d.s; ++b)
                for (int a = 0; a < d.s; ++a)
                    if (!solid[(size_t)(pj * d.s + b) * d.nxc + pi * d.s + a]) fluid = true;
            if (!fluid) continue;
            if (id) (*id)[(size_t)pj * npx + pi] = P;
            if (cell) cell->push_back(pj * npx + pi);
            ++P;
        }
    return P;
}

int validate_desc(const dnnmg_mesh_desc *d) {
    if (!d) return fail(DNNMG_EINVAL, "mesh description is NULL");
    if (d->nxc <= 0 || d->nyc <= 0 || d->nxc % 2 || d->nyc % 2)
        return fail(DNNMG_EINVAL, "nxc=%d, nyc=%d: cell counts must be positive and even", d->nxc, d->nyc);
    if (d->K < 1 || d->K > 3) return fail(DNNMG_EINVAL, "K=%d out of range 1..3", d->K);
    if (d->s < 1 || d->s > 2) return fail(DNNMG_EINVAL, "s=%d out of range 1..2", d->s);
    if (d->nxc % d->s || d->nyc % d->s)
        return fail(DNNMG_EINVAL, "patch size s=%d must divide nxc=%d and nyc=%d", d->s, d->nxc, d->nyc);
    if (!(d->lx > 0) || !(d->ly > 0) || !(d->nu > 0) || !(d->k > 0) || !(d->alpha0 >= 0))
        return fail(DNNMG_EINVAL, "lx, ly, nu, k must be > 0 and alpha0 >= 0");
    if (d->precision < DNNMG_F64 || d->precision > DNNMG_BF16NET)
        return fail(DNNMG_EINVAL, "unknown precision %d", d->precision);
    const long long nyf = (long long)d->nyc << d->K, nxf = (long long)d->nxc << d->K;
    if (nyf + 1 > 65535) return fail(DNNMG_EUNSUPPORTED, "nyf=%lld: at most 65534 fine rows", nyf);
    if ((nxf + 64) * (nyf + 1) > (1LL << 31))
        return fail(DNNMG_EUNSUPPORTED, "%lld fine nodes: at most 2^31", (nxf + 1) * (nyf + 1));
    const int S = d->s << d->K, n_in = 3 * (S + 1) * (S + 1) + 3 * (d->s + 1) * (d->s + 1) + 12;
    if (round_up(n_in, 16) > feature_table_capacity())
        return fail(DNNMG_EUNSUPPORTED, "%d network inputs: at most %d", n_in, feature_table_capacity());
    return DNNMG_OK;
}

void fill_info(const dnnmg_mesh_desc &d, int P, int n_solid, dnnmg_mesh_info *info) {
    dnnmg_mesh_info &I = *info;
    memset(&I, 0, sizeof I);
    I.nxc = d.nxc;
    I.nyc = d.nyc;
    I.K = d.K;
    I.s = d.s;
    I.nxf = d.nxc << d.K;
    I.nyf = d.nyc << d.K;
    I.npx = d.nxc / d.s;
    I.npy = d.nyc / d.s;
    I.Nc = (long long)(d.nxc + 1) * (d.nyc + 1);
    I.Nf = (long long)(I.nxf + 1) * (I.nyf + 1);
    I.pitch = round_up(I.nxf + 1, 64);
    I.plane = (long long)I.pitch * (I.nyf + 1);
    I.P = P;
    const int S = d.s << d.K;
    I.nf = (S + 1) * (S + 1);
    I.nc = (d.s + 1) * (d.s + 1);
    I.n_in = 3 * I.nf + 3 * I.nc + 12;
    I.n_out = 2 * I.nf;
    I.ldx = round_up(I.n_in, 16);
    I.n_solid_coarse = n_solid;
    I.precision = d.precision;
    I.real_bytes = d.precision == DNNMG_F64 ? 8 : 4;
    I.feature_bytes = d.precision == DNNMG_F64 ? 8 : (d.precision == DNNMG_F32 ? 4 : 2);
    size_t ws = 0;
    ws += align256((size_t)P * I.ldx * I.feature_bytes);        // X
    ws += align256((size_t)P * I.n_out * I.real_bytes);         // d
    ws += align256(2 * (size_t)I.plane * I.real_bytes);         // v_corr
    ws += align256(3 * (size_t)(d.nyc + 1) * round_up(d.nxc + 1, 32) * I.real_bytes);   // padded x_c
    ws += 2 * align256(3 * (size_t)I.Nc * sizeof(double));      // host-call staging of x_c, b_c
    I.workspace_bytes = ws;
}

struct Workspace {
    void *X, *d, *vc, *xcp;
    double *xc, *bc;
};

Workspace carve(const dnnmg_mesh_info &I, void *base) {
    Workspace w;
    char *p = static_cast<char *>(base);
    w.X = p;
    p += align256((size_t)I.P * I.ldx * I.feature_bytes);
    w.d = p;
    p += align256((size_t)I.P * I.n_out * I.real_bytes);
    w.vc = p;
    p += align256(2 * (size_t)I.plane * I.real_bytes);
    w.xcp = p;
    p += align256(3 * (size_t)(I.nyc + 1) * round_up(I.nxc + 1, 32) * I.real_bytes);
    w.xc = reinterpret_cast<double *>(p);
    p += align256(3 * (size_t)I.Nc * sizeof(double));
    w.bc = reinterpret_cast<double *>(p);
    return w;
}

// Element matrices of a fine hx x hy cell from 1D linear factors, the 2x2
// Gauss tables for the convection term, and the LPS patch matrix.
void fem_coefficients(const dnnmg_mesh_desc &d, FemCoef<double> *out) {
    FemCoef<double> &f = *out;
    memset(&f, 0, sizeof f);
    const double hx = d.lx / (d.nxc << d.K), hy = d.ly / (d.nyc << d.K);
    double M1x[2][2], M1y[2][2], K1x[2][2], K1y[2][2], C1x[2][2], C1y[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            M1x[a][b] = hx / 6.0 * (a == b ? 2.0 : 1.0);
            M1y[a][b] = hy / 6.0 * (a == b ? 2.0 : 1.0);
            K1x[a][b] = (a == b ? 1.0 : -1.0) / hx;
            K1y[a][b] = (a == b ? 1.0 : -1.0) / hy;
            C1x[a][b] = a == 0 ? -0.5 : 0.5;   // int l_b l_a' over the 1D cell
            C1y[a][b] = a == 0 ? -0.5 : 0.5;
        }
    double Kd[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const int ax = a & 1, ay = a >> 1, bx = b & 1, by = b >> 1;
            const double M = M1x[ax][bx] * M1y[ay][by];
            Kd[a][b] = K1x[ax][bx] * M1y[ay][by] + M1x[ax][bx] * K1y[ay][by];
            f.Av[a][b] = M / d.k + 0.5 * d.nu * Kd[a][b];
            f.Bv[a][b] = M / d.k - 0.5 * d.nu * Kd[a][b];
            f.Gx[a][b] = C1x[ax][bx] * M1y[ay][by];
            f.Gy[a][b] = M1x[ax][bx] * C1y[ay][by];
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            f.Dx[a][b] = f.Gx[b][a];
            f.Dy[a][b] = f.Gy[b][a];
        }
    const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    for (int qy = 0; qy < 2; ++qy)
        for (int qx = 0; qx < 2; ++qx) {
            const int q = 2 * qy + qx;
            const double xi = gp[qx], eta = gp[qy];
            const double lx[2] = {1 - xi, xi}, ly[2] = {1 - eta, eta}, dl[2] = {-1.0, 1.0};
            for (int a = 0; a < 4; ++a) {
                const int ax = a & 1, ay = a >> 1;
                f.qphi[q][a] = lx[ax] * ly[ay];
                f.qdx[q][a] = dl[ax] * ly[ay] / hx;
                f.qdy[q][a] = lx[ax] * dl[ay] / hy;
            }
        }
    f.qw = hx * hy / 4.0;
    // LPS on a 2x2-cell patch: S9 = alpha (I - Pi)^T L (I - Pi)
    double L[9][9] = {}, Pi[9][9] = {}, Q[9][9], T1[9][9];
    for (int cb = 0; cb < 2; ++cb)
        for (int ca = 0; ca < 2; ++ca) {
            const int idx[4] = {3 * cb + ca, 3 * cb + ca + 1, 3 * (cb + 1) + ca, 3 * (cb + 1) + ca + 1};
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) L[idx[a]][idx[b]] += Kd[a][b];
        }
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            const double X = a / 2.0, Y = b / 2.0;
            Pi[3 * b + a][0] += (1 - X) * (1 - Y);
            Pi[3 * b + a][2] += X * (1 - Y);
            Pi[3 * b + a][6] += (1 - X) * Y;
            Pi[3 * b + a][8] += X * Y;
        }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) Q[i][j] = (i == j ? 1.0 : 0.0) - Pi[i][j];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0;
            for (int k = 0; k < 9; ++k) s += L[i][k] * Q[k][j];
            T1[i][j] = s;
        }
    const double alpha = d.alpha0 * (hx * hx + hy * hy) / d.nu;
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0;
            for (int k = 0; k < 9; ++k) s += Q[k][i] * T1[k][j];
            f.S9[i][j] = alpha * s;
        }
    // patch geometry from its corners: edges, aspect ratios, angles
    const double w = d.s * (d.lx / d.nxc), h = d.s * (d.ly / d.nyc);
    const double cx[4] = {0, w, w, 0}, cy[4] = {0, 0, h, h};   // SW, SE, NE, NW
    double len[4];
    for (int e = 0; e < 4; ++e) len[e] = std::hypot(cx[(e + 1) % 4] - cx[e], cy[(e + 1) % 4] - cy[e]);
    f.geo[0] = len[0];
    f.geo[1] = len[1];
    f.geo[2] = len[2];
    f.geo[3] = len[3];
    f.geo[4] = len[0] / len[1];
    f.geo[5] = len[2] / len[3];
    f.geo[6] = len[0] / len[2];
    f.geo[7] = len[3] / len[1];
    for (int c = 0; c < 4; ++c) {
        const int n = (c + 1) % 4, p = (c + 3) % 4;
        const double ax = cx[n] - cx[c], ay = cy[n] - cy[c], bx = cx[p] - cx[c], by = cy[p] - cy[c];
        f.geo[8 + c] = std::acos((ax * bx + ay * by) / (std::hypot(ax, ay) * std::hypot(bx, by)));
    }
    f.q_over_nu = d.s * std::fmax(d.lx / d.nxc, d.ly / d.nyc) / d.nu;
    // node stencils: sum the element rows of the 4 cells around a node
    auto stencil = [](const double E[4][4], double S[3][3]) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] = 0.0;
        for (int cy = -1; cy <= 0; ++cy)
            for (int cx = -1; cx <= 0; ++cx) {
                const int a = -cx + 2 * (-cy);
                for (int b = 0; b < 4; ++b) S[cy + (b >> 1) + 1][cx + (b & 1) + 1] += E[a][b];
            }
    };
    stencil(f.Av, f.nA);
    stencil(f.Bv, f.nB);
    stencil(f.Gx, f.nGx);
    stencil(f.Gy, f.nGy);
    stencil(f.Dx, f.nDx);
    stencil(f.Dy, f.nDy);
    for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px)
            for (int ey = 0; ey < 2 - py; ++ey)
                for (int ex = 0; ex < 2 - px; ++ex) {
                    const int a = px ? 1 : 2 * ex, b = py ? 1 : 2 * ey;   // the node in this patch
                    for (int kb = 0; kb < 3; ++kb)
                        for (int ka = 0; ka < 3; ++ka)
                            f.L5[py][px][kb - b + 2][ka - a + 2] += f.S9[3 * b + a][3 * kb + ka];
                }
    f.cg0 = gp[0];
    f.cg1 = gp[1];
    f.inv_hx = 1.0 / hx;
    f.inv_hy = 1.0 / hy;
    f.cwg0 = 0.5 * f.qw * gp[0];
    f.cwg1 = 0.5 * f.qw * gp[1];
    (void)kPi;
}

void to_float(const FemCoef<double> &a, FemCoef<float> *b) {
    const double *src = reinterpret_cast<const double *>(&a);
    float *dst = reinterpret_cast<float *>(b);
    static_assert(sizeof(FemCoef<double>) == 2 * sizeof(FemCoef<float>), "layout");
    for (size_t i = 0; i < sizeof(FemCoef<float>) / sizeof(float); ++i) dst[i] = (float)src[i];
}

int check_device(int dev) {
    int cur = -1;
    DNNMG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev)
        return fail(DNNMG_EINVAL, "handle belongs to device %d but device %d is current", dev, cur);
    return DNNMG_OK;
}

bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

int check_mesh(dnnmg_mesh_t m) {
    if (!m) return fail(DNNMG_EINVAL, "mesh handle is NULL");
    return check_device(m->device);
}

}  // namespace
}  // namespace dnnmg

namespace dnnmg {
// Element constants of a single uniform level of nx x ny cells (the
// multigrid levels): the same construction as a mesh's fine level.
void level_coefficients(double lx, double ly, int nx, int ny, double nu, double k, double alpha0,
                        FemCoef<double> *f64, FemCoef<float> *f32) {
    dnnmg_mesh_desc d;
    memset(&d, 0, sizeof d);
    d.nxc = nx;
    d.nyc = ny;
    d.K = 0;
    d.s = 1;
    d.lx = lx;
    d.ly = ly;
    d.nu = nu;
    d.k = k;
    d.alpha0 = alpha0;
    fem_coefficients(d, f64);
    to_float(*f64, f32);
}
}  // namespace dnnmg

using namespace dnnmg;

extern "C" {

const char *dnnmg_last_error(void) { return g_error.c_str(); }

int dnnmg_mesh_query(const dnnmg_mesh_desc *desc, dnnmg_mesh_info *info) {
    clear_error();
    if (int e = validate_desc(desc)) return e;
    if (!info) return fail(DNNMG_EINVAL, "info is NULL");
    std::vector<uint8_t> solid = solid_mask(*desc);
    int n_solid = 0;
    for (uint8_t v : solid) n_solid += v;
    const int P = patch_numbering(*desc, solid, nullptr, nullptr);
    fill_info(*desc, P, n_solid, info);
    return DNNMG_OK;
}

int dnnmg_mesh_create(const dnnmg_mesh_desc *desc, dnnmg_mesh_t *out) {
    clear_error();
    if (int e = validate_desc(desc)) return e;
    if (!out) return fail(DNNMG_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<uint8_t> solid = solid_mask(*desc);
    std::vector<int> pid, pcell;
    int n_solid = 0;
    for (uint8_t v : solid) n_solid += v;
    const int P = patch_numbering(*desc, solid, &pid, &pcell);
    dnnmg_mesh_s *m = new (std::nothrow) dnnmg_mesh_s();
    if (!m) return fail(DNNMG_ENOMEM, "host allocation failed");
    m->desc = *desc;
    m->desc.solid = nullptr;
    fill_info(*desc, P, n_solid, &m->info);
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return fail(DNNMG_ECUDA, "cudaGetDevice failed");
    }
    m->d_solid = nullptr;
    m->d_patch_id = nullptr;
    m->d_patch_cell = nullptr;
    const size_t ns = solid.size(), np = pid.size(), nc = pcell.size();
    if (cudaMalloc(&m->d_solid, ns) != cudaSuccess ||
        cudaMalloc(&m->d_patch_id, np * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&m->d_patch_cell, (nc ? nc : 1) * sizeof(int)) != cudaSuccess) {
        cudaFree(m->d_solid);
        cudaFree(m->d_patch_id);
        cudaFree(m->d_patch_cell);
        delete m;
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the mesh maps failed");
    }
    if (cudaMemcpy(m->d_solid, solid.data(), ns, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->d_patch_id, pid.data(), np * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        (nc && cudaMemcpy(m->d_patch_cell, pcell.data(), nc * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)) {
        cudaFree(m->d_solid);
        cudaFree(m->d_patch_id);
        cudaFree(m->d_patch_cell);
        delete m;
        return fail(DNNMG_ECUDA, "upload of the mesh maps failed");
    }
    MeshGeom &g = m->g;
    const dnnmg_mesh_info &I = m->info;
    g.nxc = I.nxc; g.nyc = I.nyc; g.K = I.K; g.r = 1 << I.K; g.s = I.s; g.S = I.s << I.K;
    g.nxf = I.nxf; g.nyf = I.nyf; g.npx = I.npx; g.npy = I.npy; g.P = P;
    g.pitch = I.pitch; g.plane = (size_t)I.plane;
    g.nf = I.nf; g.nc = I.nc; g.n_in = I.n_in; g.n_out = I.n_out; g.ldx = I.ldx;
    g.lx = desc->lx; g.ly = desc->ly;
    g.hxc = desc->lx / I.nxc; g.hyc = desc->ly / I.nyc;
    g.hxf = desc->lx / I.nxf; g.hyf = desc->ly / I.nyf;
    g.nu = desc->nu; g.k = desc->k; g.u_max = desc->u_max; g.ramp = desc->ramp;
    g.solid = m->d_solid;
    g.patch_id = m->d_patch_id;
    g.patch_cell = m->d_patch_cell;
    std::vector<int> tab((size_t)I.ldx);
    feature_table(g, tab.data());
    m->d_feat_tab = nullptr;
    if (cudaMalloc(&m->d_feat_tab, tab.size() * sizeof(int)) != cudaSuccess ||
        cudaMemcpy(m->d_feat_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(m->d_solid);
        cudaFree(m->d_patch_id);
        cudaFree(m->d_patch_cell);
        cudaFree(m->d_feat_tab);
        delete m;
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the feature table failed");
    }
    g.feat_tab = m->d_feat_tab;
    tile_counts(g, &g.ntx, &g.nty);
    std::vector<uint8_t> tflags((size_t)g.ntx * g.nty);
    tile_flags(g, solid.data(), tflags.data());
    m->d_tile_flags = nullptr;
    if (cudaMalloc(&m->d_tile_flags, tflags.size()) != cudaSuccess ||
        cudaMemcpy(m->d_tile_flags, tflags.data(), tflags.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(m->d_solid);
        cudaFree(m->d_patch_id);
        cudaFree(m->d_patch_cell);
        cudaFree(m->d_feat_tab);
        cudaFree(m->d_tile_flags);
        delete m;
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the tile flags failed");
    }
    g.tile_flags = m->d_tile_flags;
    auto undo = [&](const char *what) {
        if (m->side) cudaStreamDestroy(m->side);
        if (m->ev_fork) cudaEventDestroy(m->ev_fork);
        if (m->ev_join) cudaEventDestroy(m->ev_join);
        cudaFree(m->d_solid);
        cudaFree(m->d_patch_id);
        cudaFree(m->d_patch_cell);
        cudaFree(m->d_feat_tab);
        cudaFree(m->d_tile_flags);
        cudaFree(m->d_slow_tiles);
        cudaFree(m->d_cf_tab);
        cudaFree(m->d_status);
        delete m;
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the %s failed", what);
    };
    // tiles the general S2+S3 kernel does when the all-fluid ones run in closed form
    std::vector<int> slow;
    residual_cf_slow_tiles(g, tflags.data(), &slow);
    g.n_slow_tiles = (int)slow.size();
    m->d_slow_tiles = nullptr;
    if (cudaMalloc(&m->d_slow_tiles, (slow.size() ? slow.size() : 1) * sizeof(int)) != cudaSuccess ||
        (slow.size() && cudaMemcpy(m->d_slow_tiles, slow.data(), slow.size() * sizeof(int),
                                   cudaMemcpyHostToDevice) != cudaSuccess))
        return undo("boundary tile list");
    g.slow_tiles = m->d_slow_tiles;
    std::vector<uint16_t> ctab((size_t)I.ldx);
    residual_cf_table(g, ctab.data());
    m->d_cf_tab = nullptr;
    if (cudaMalloc(&m->d_cf_tab, ctab.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMemcpy(m->d_cf_tab, ctab.data(), ctab.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return undo("closed-form column table");
    g.cf_tab = m->d_cf_tab;
    m->d_status = nullptr;
    if (cudaMalloc(&m->d_status, sizeof(int)) != cudaSuccess || cudaMemset(m->d_status, 0, sizeof(int)) != cudaSuccess)
        return undo("mesh status");
    g.status = m->d_status;
    if (cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return undo("side stream and its events");
    fem_coefficients(*desc, &m->fem64);
    to_float(m->fem64, &m->fem32);
    *out = m;
    return DNNMG_OK;
}

int dnnmg_mesh_destroy(dnnmg_mesh_t mesh) {
    clear_error();
    if (!mesh) return DNNMG_OK;
    cudaFree(mesh->d_solid);
    cudaFree(mesh->d_patch_id);
    cudaFree(mesh->d_patch_cell);
    cudaFree(mesh->d_feat_tab);
    cudaFree(mesh->d_tile_flags);
    cudaFree(mesh->d_slow_tiles);
    cudaFree(mesh->d_cf_tab);
    cudaFree(mesh->d_status);
    if (mesh->side) cudaStreamDestroy(mesh->side);
    if (mesh->ev_fork) cudaEventDestroy(mesh->ev_fork);
    if (mesh->ev_join) cudaEventDestroy(mesh->ev_join);
    delete mesh;
    return DNNMG_OK;
}

int dnnmg_mesh_get_info(dnnmg_mesh_t mesh, dnnmg_mesh_info *info) {
    clear_error();
    if (!mesh || !info) return fail(DNNMG_EINVAL, "NULL argument");
    *info = mesh->info;
    return DNNMG_OK;
}

int dnnmg_mesh_maps(dnnmg_mesh_t mesh, int *patch_cell, unsigned char *node_flags,
                    unsigned char *node_mult, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (patch_cell && mesh->info.P)
        DNNMG_CUDA_TRY(cudaMemcpyAsync(patch_cell, mesh->d_patch_cell, sizeof(int) * mesh->info.P,
                                       cudaMemcpyDeviceToDevice, stream));
    if (node_flags || node_mult) {
        DNNMG_CUDA_TRY(launch_mesh_maps(mesh->g, node_flags, node_mult, stream));
    }
    return DNNMG_OK;
}

int dnnmg_net_create(int n_in, int hidden, int n_out, const double *Wx, const double *Uh,
                     const double *Wfc, int precision, dnnmg_net_t *out) {
    clear_error();
    if (!out || !Wx || !Uh || !Wfc) return fail(DNNMG_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_in <= 0 || hidden <= 0 || n_out <= 0 || n_in > 4096 || hidden > 1024 || n_out > 4096)
        return fail(DNNMG_EINVAL, "network sizes n_in=%d H=%d n_out=%d out of range", n_in, hidden, n_out);
    if (precision < DNNMG_F64 || precision > DNNMG_BF16NET)
        return fail(DNNMG_EINVAL, "unknown precision %d", precision);
    dnnmg_net_s *n = new (std::nothrow) dnnmg_net_s();
    if (!n) return fail(DNNMG_ENOMEM, "host allocation failed");
    n->n_in = n_in;
    n->ldx = round_up(n_in, 16);
    n->H = hidden;
    n->n_out = n_out;
    n->precision = precision;
    n->WxT = n->UhT = n->WfcT = n->tc_weights = nullptr;
    n->tc = nullptr;
    n->d_status = nullptr;
    n->tc_bytes = 0;
    cudaGetDevice(&n->device);
    if (cudaMalloc(&n->d_status, sizeof(int)) != cudaSuccess || cudaMemset(n->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(n->d_status);
        delete n;
        cudaGetLastError();
        return fail(DNNMG_ENOMEM, "device allocation of the status word failed");
    }
    const int G = 3 * hidden;
    std::vector<double> wx((size_t)n->ldx * G, 0.0), uh((size_t)hidden * G), wfc((size_t)hidden * n_out);
    for (int j = 0; j < G; ++j)
        for (int k = 0; k < n_in; ++k) wx[(size_t)k * G + j] = Wx[(size_t)j * n_in + k];
    for (int j = 0; j < G; ++j)
        for (int k = 0; k < hidden; ++k) uh[(size_t)k * G + j] = Uh[(size_t)j * hidden + k];
    for (int o = 0; o < n_out; ++o)
        for (int k = 0; k < hidden; ++k) wfc[(size_t)k * n_out + o] = Wfc[(size_t)o * hidden + k];
    auto upload = [&](const std::vector<double> &src, void **dst) -> int {
        const size_t cnt = src.size();
        if (precision == DNNMG_F64) {
            if (cudaMalloc(dst, cnt * 8) != cudaSuccess) return DNNMG_ENOMEM;
            return cudaMemcpy(*dst, src.data(), cnt * 8, cudaMemcpyHostToDevice) == cudaSuccess ? 0 : DNNMG_ECUDA;
        }
        if (precision == DNNMG_F32) {
            std::vector<float> t(src.begin(), src.end());
            if (cudaMalloc(dst, cnt * 4) != cudaSuccess) return DNNMG_ENOMEM;
            return cudaMemcpy(*dst, t.data(), cnt * 4, cudaMemcpyHostToDevice) == cudaSuccess ? 0 : DNNMG_ECUDA;
        }
        std::vector<__nv_bfloat16> t(cnt);
        for (size_t i = 0; i < cnt; ++i) t[i] = __float2bfloat16_rn((float)src[i]);
        if (cudaMalloc(dst, cnt * 2) != cudaSuccess) return DNNMG_ENOMEM;
        return cudaMemcpy(*dst, t.data(), cnt * 2, cudaMemcpyHostToDevice) == cudaSuccess ? 0 : DNNMG_ECUDA;
    };
    int e = upload(wx, &n->WxT);
    if (!e) e = upload(uh, &n->UhT);
    if (!e) e = upload(wfc, &n->WfcT);
    if (e) {
        cudaFree(n->WxT);
        cudaFree(n->UhT);
        cudaFree(n->WfcT);
        cudaFree(n->d_status);
        delete n;
        cudaGetLastError();
        return fail(e, "uploading the network weights failed");
    }
    // BF16 networks run on the tensor cores when the shapes allow it;
    // DNNMG_GRU_KERNEL=simt selects the CUDA-core kernel (same arithmetic).
    const char *which = getenv("DNNMG_GRU_KERNEL");
    if (precision == DNNMG_BF16NET && !(which && strcmp(which, "simt") == 0)) {
        if (!tc_prepare(*n, Wx, Uh, Wfc)) cudaGetLastError();
    }
    *out = n;
    return DNNMG_OK;
}

int dnnmg_net_destroy(dnnmg_net_t net) {
    clear_error();
    if (!net) return DNNMG_OK;
    cudaFree(net->WxT);
    cudaFree(net->UhT);
    cudaFree(net->WfcT);
    cudaFree(net->tc_weights);
    cudaFree(net->d_status);
    tc_release(*net);
    delete net;
    return DNNMG_OK;
}

int dnnmg_prolongate(dnnmg_mesh_t mesh, const double *xc, void *xf, double t, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (!xc || !xf) return fail(DNNMG_EINVAL, "NULL array");
    if (!aligned16(xf)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_prolongate(mesh->g, mesh->info.precision, xc, xf, t, stream));
    return DNNMG_OK;
}

int dnnmg_patch_features(dnnmg_mesh_t mesh, const void *xf, const double *xc, double t, const void *bf,
                         void *rf, void *X, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (!bf || (!X && mesh->info.P)) return fail(DNNMG_EINVAL, "NULL array");
    if ((xf == nullptr) == (xc == nullptr)) return fail(DNNMG_EINVAL, "exactly one of xf and xc must be given");
    if ((xf && !aligned16(xf)) || !aligned16(bf) || (rf && !aligned16(rf)))
        return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_residual_features(mesh->g, mesh->info.precision, mesh->fem64, mesh->fem32,
                                            xf, xc, t, bf, rf, X, stream));
    return DNNMG_OK;
}

int dnnmg_gru_step(dnnmg_net_t net, const void *X, void *h, void *d, int P, cudaStream_t stream) {
    clear_error();
    if (!net) return fail(DNNMG_EINVAL, "net handle is NULL");
    if (int e = check_device(net->device)) return e;
    if (P < 0) return fail(DNNMG_EINVAL, "P=%d < 0", P);
    if (P == 0) return DNNMG_OK;
    if (!X || !h || !d) return fail(DNNMG_EINVAL, "NULL array");
    if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(h) % 16 ||
        reinterpret_cast<uintptr_t>(d) % 16)
        return fail(DNNMG_EINVAL, "X, h and d must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_gru(*net, X, h, d, P, stream));
    return DNNMG_OK;
}

int dnnmg_scatter_avg(dnnmg_mesh_t mesh, const void *d, const void *xf, const double *xc, double t,
                      void *vcorr, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if ((!d && mesh->info.P) || !vcorr) return fail(DNNMG_EINVAL, "NULL array");
    if ((xf == nullptr) == (xc == nullptr)) return fail(DNNMG_EINVAL, "exactly one of xf and xc must be given");
    if ((xf && !aligned16(xf)) || !aligned16(vcorr)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_scatter_avg(mesh->g, mesh->info.precision, d, xf, xc, t, vcorr, stream));
    return DNNMG_OK;
}

int dnnmg_rhs_restrict(dnnmg_mesh_t mesh, const void *vcorr, void *bf, double *bc,
                       cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (!vcorr || !bf || !bc) return fail(DNNMG_EINVAL, "NULL array");
    if (vcorr == bf) return fail(DNNMG_EINVAL, "vcorr and bf must not alias");
    if (!aligned16(vcorr) || !aligned16(bf)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_rhs(mesh->g, mesh->info.precision, mesh->fem64, mesh->fem32, vcorr, bf, stream));
    DNNMG_CUDA_TRY(launch_restrict(mesh->g, mesh->info.precision, bf, bc, stream));
    return DNNMG_OK;
}

int dnnmg_rhs(dnnmg_mesh_t mesh, const void *vcorr, void *bf, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (!vcorr || !bf) return fail(DNNMG_EINVAL, "NULL array");
    if (vcorr == bf) return fail(DNNMG_EINVAL, "vcorr and bf must not alias");
    if (!aligned16(vcorr) || !aligned16(bf)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_rhs(mesh->g, mesh->info.precision, mesh->fem64, mesh->fem32, vcorr, bf, stream));
    return DNNMG_OK;
}

int dnnmg_scatter_rhs(dnnmg_mesh_t mesh, const void *d, const double *xc, double t, void *bf,
                      cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if ((!d && mesh->info.P) || !xc || !bf) return fail(DNNMG_EINVAL, "NULL array");
    if (!aligned16(bf)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(d) % 8) return fail(DNNMG_EINVAL, "d must be 8-byte aligned");
    DNNMG_CUDA_TRY(launch_avg_rhs(mesh->g, mesh->info.precision, mesh->fem64, mesh->fem32, d, xc, t, bf, stream));
    return DNNMG_OK;
}

int dnnmg_restrict(dnnmg_mesh_t mesh, const void *bf, double *bc, cudaStream_t stream) {
    clear_error();
    if (int e = check_mesh(mesh)) return e;
    if (!bf || !bc) return fail(DNNMG_EINVAL, "NULL array");
    if (!aligned16(bf)) return fail(DNNMG_EINVAL, "fine fields must be 16-byte aligned");
    DNNMG_CUDA_TRY(launch_restrict(mesh->g, mesh->info.precision, bf, bc, stream));
    return DNNMG_OK;
}

int dnnmg_net_status(dnnmg_net_t net, int *status, int reset) {
    clear_error();
    if (!net || !status) return fail(DNNMG_EINVAL, "NULL argument");
    if (int e = check_device(net->device)) return e;
    DNNMG_CUDA_TRY(cudaMemcpy(status, net->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset) DNNMG_CUDA_TRY(cudaMemset(net->d_status, 0, sizeof(int)));
    return DNNMG_OK;
}

int dnnmg_net_uses_tensor_cores(dnnmg_net_t net) { return net && net->tc ? 1 : 0; }

int dnnmg_mesh_status(dnnmg_mesh_t mesh, int *status, int reset) {
    clear_error();
    if (!mesh || !status) return fail(DNNMG_EINVAL, "NULL argument");
    if (int e = check_device(mesh->device)) return e;
    DNNMG_CUDA_TRY(cudaMemcpy(status, mesh->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset) DNNMG_CUDA_TRY(cudaMemset(mesh->d_status, 0, sizeof(int)));
    return DNNMG_OK;
}

// Bytes of the workspace that the device-buffer step uses: all of it but the
// staging of x_c and b_c, which only dnnmg_step_host's pageable path needs.
static size_t device_step_bytes(const dnnmg_mesh_info &I) {
    return I.workspace_bytes - 2 * align256(3 * (size_t)I.Nc * sizeof(double));
}

static int step_checks(dnnmg_mesh_t mesh, dnnmg_net_t net, void *h, void *bf, void *workspace,
                       size_t workspace_bytes, bool device_only = false) {
    if (int e = check_mesh(mesh)) return e;
    if (!net) return fail(DNNMG_EINVAL, "net handle is NULL");
    const dnnmg_mesh_info &I = mesh->info;
    if (net->n_in != I.n_in || net->n_out != I.n_out)
        return fail(DNNMG_EINVAL, "network is %d -> %d but the mesh needs %d -> %d", net->n_in,
                    net->n_out, I.n_in, I.n_out);
    if (net->precision != I.precision)
        return fail(DNNMG_EINVAL, "network precision %d differs from mesh precision %d",
                    net->precision, I.precision);
    // h has P rows: a mesh without fluid patches has no state
    if ((!h && I.P > 0) || !bf || !workspace) return fail(DNNMG_EINVAL, "NULL array");
    if (!aligned16(bf) || !aligned16(h)) return fail(DNNMG_EINVAL, "bf and h must be 16-byte aligned");
    const size_t need = device_only ? device_step_bytes(I) : I.workspace_bytes;
    if (workspace_bytes < need) return fail(DNNMG_EINVAL, "workspace of %zu bytes, %zu needed", workspace_bytes, need);
    if (reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(DNNMG_EINVAL, "workspace must be 256-byte aligned");
    return DNNMG_OK;
}

// ev (may be null): dnnmg_step_launches() + 1 events, recorded before the
// first kernel and after each kernel.
static int step_body(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf,
                     double *bc, const Workspace &w, double t, cudaStream_t s, cudaEvent_t *ev = nullptr) {
    const int prec = mesh->info.precision;
    const MeshGeom &g = mesh->g;
    int nev = 0;
    auto mark = [&]() -> cudaError_t { return ev ? cudaEventRecord(ev[nev++], s) : cudaSuccess; };
    DNNMG_CUDA_TRY(mark());
    // S1 is fused into S2+S3 and into S5: both interpolate x~ from xc inside
    // their tiles, so x~ never goes to memory; S2+S3 reads x_c as a padded
    // copy in the fine type, fetched by TMA.  (S5+S6 as one kernel keeps
    // v_corr on chip but averages every tile's halo again and waits on two
    // dependent global fetches per tile; it measured slower than the v_corr
    // round trip.  See dnnmg_scatter_rhs.)
    DNNMG_CUDA_TRY(launch_coarse_pad(g, prec, xc, w.xcp, s));
    DNNMG_CUDA_TRY(mark());
    // S2 + S3: all-fluid tiles in closed form (x~ = P x_c is bilinear per
    // coarse cell there), the other tiles by the general element kernel
    const bool cf = residual_cf_supported(g, prec);
    if (cf && !ev && g.n_slow_tiles > 0) {
        // the two S2+S3 kernels write disjoint rows of X: the boundary tiles
        // (few, slow CTAs) run on the side stream while the closed form runs
        DNNMG_CUDA_TRY(cudaEventRecord(mesh->ev_fork, s));
        DNNMG_CUDA_TRY(cudaStreamWaitEvent(mesh->side, mesh->ev_fork, 0));
        DNNMG_CUDA_TRY(launch_residual_step(g, prec, mesh->fem64, mesh->fem32, w.xcp, t, bf, w.X, mesh->side, true));
        DNNMG_CUDA_TRY(launch_residual_cf(g, prec, mesh->fem32, w.xcp, bf, w.X, s));
        DNNMG_CUDA_TRY(cudaEventRecord(mesh->ev_join, mesh->side));
        DNNMG_CUDA_TRY(cudaStreamWaitEvent(s, mesh->ev_join, 0));
    } else {
        // (the timed form runs them one after the other, to time each)
        if (cf) {
            DNNMG_CUDA_TRY(launch_residual_cf(g, prec, mesh->fem32, w.xcp, bf, w.X, s));
            DNNMG_CUDA_TRY(mark());
        }
        DNNMG_CUDA_TRY(launch_residual_step(g, prec, mesh->fem64, mesh->fem32, w.xcp, t, bf, w.X, s, cf));
        DNNMG_CUDA_TRY(mark());
    }
    if (mesh->info.P) {
        DNNMG_CUDA_TRY(launch_gru(*net, w.X, h, w.d, mesh->info.P, s));
        DNNMG_CUDA_TRY(mark());
    }
    DNNMG_CUDA_TRY(launch_scatter_avg(g, prec, w.d, nullptr, xc, t, w.vc, s, w.xcp));
    DNNMG_CUDA_TRY(mark());
    DNNMG_CUDA_TRY(launch_rhs(g, prec, mesh->fem64, mesh->fem32, w.vc, bf, s));
    DNNMG_CUDA_TRY(mark());
    DNNMG_CUDA_TRY(launch_restrict(g, prec, bf, bc, s));
    DNNMG_CUDA_TRY(mark());
    return DNNMG_OK;
}

}  // extern "C"

namespace dnnmg {
size_t step_scratch_bytes(const dnnmg_mesh_info &I) { return device_step_bytes(I); }

// dnnmg_step with the checks done on the given scratch (used by step_static.cu):
// the scratch needs only the device step's part of a workspace.
int step_on_workspace(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
                      void *workspace, size_t workspace_bytes, double t, cudaStream_t stream) {
    if (int e = step_checks(mesh, net, h, bf, workspace, workspace_bytes, true)) return e;
    if (!xc || !bc) return fail(DNNMG_EINVAL, "NULL array");
    return step_body(mesh, net, xc, h, bf, bc, carve(mesh->info, workspace), t, stream);
}
}  // namespace dnnmg

extern "C" {

int dnnmg_step(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
               void *workspace, size_t workspace_bytes, double t, cudaStream_t stream) {
    clear_error();
    if (int e = step_checks(mesh, net, h, bf, workspace, workspace_bytes)) return e;
    if (!xc || !bc) return fail(DNNMG_EINVAL, "NULL array");
    return step_body(mesh, net, xc, h, bf, bc, carve(mesh->info, workspace), t, stream);
}

int dnnmg_step_host(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc_host, void *h, void *bf,
                    double *bc_host, void *workspace, size_t workspace_bytes, double t,
                    cudaStream_t stream) {
    clear_error();
    if (int e = step_checks(mesh, net, h, bf, workspace, workspace_bytes)) return e;
    if (!xc_host || !bc_host) return fail(DNNMG_EINVAL, "NULL array");
    const Workspace w = carve(mesh->info, workspace);
    // Page-locked (mapped) host buffers are read and written by the step's
    // kernels directly over the CPU-GPU link: x_c only by the coarse copy
    // (the averaging reads the padded copy), b_c only by the restriction.
    auto mapped = [](const void *p) -> void * {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    };
    const double *xc_dev = static_cast<const double *>(mapped(xc_host));
    double *bc_dev = static_cast<double *>(mapped(bc_host));
    if (xc_dev && bc_dev) return step_body(mesh, net, xc_dev, h, bf, bc_dev, w, t, stream);
    const size_t nbytes = 3 * (size_t)mesh->info.Nc * sizeof(double);
    DNNMG_CUDA_TRY(cudaMemcpyAsync(w.xc, xc_host, nbytes, cudaMemcpyHostToDevice, stream));
    if (int e = step_body(mesh, net, w.xc, h, bf, w.bc, w, t, stream)) return e;
    DNNMG_CUDA_TRY(cudaMemcpyAsync(bc_host, w.bc, nbytes, cudaMemcpyDeviceToHost, stream));
    return DNNMG_OK;
}

int dnnmg_step_timed(dnnmg_mesh_t mesh, dnnmg_net_t net, const double *xc, void *h, void *bf, double *bc,
                     void *workspace, size_t workspace_bytes, double t, cudaEvent_t *events, int n_events,
                     cudaStream_t stream) {
    clear_error();
    if (int e = step_checks(mesh, net, h, bf, workspace, workspace_bytes)) return e;
    if (!xc || !bc || !events) return fail(DNNMG_EINVAL, "NULL array");
    if (n_events != dnnmg_step_launches(mesh, net) + 1)
        return fail(DNNMG_EINVAL, "%d events given, the step needs %d", n_events, dnnmg_step_launches(mesh, net) + 1);
    return step_body(mesh, net, xc, h, bf, bc, carve(mesh->info, workspace), t, stream, events);
}

int dnnmg_workspace_offsets(dnnmg_mesh_t mesh, long long *x, long long *d, long long *vcorr) {
    clear_error();
    if (!mesh || !x || !d || !vcorr) return fail(DNNMG_EINVAL, "NULL argument");
    const Workspace w = carve(mesh->info, nullptr);
    *x = static_cast<long long>(reinterpret_cast<uintptr_t>(w.X));
    *d = static_cast<long long>(reinterpret_cast<uintptr_t>(w.d));
    *vcorr = static_cast<long long>(reinterpret_cast<uintptr_t>(w.vc));
    return DNNMG_OK;
}

int dnnmg_step_launches(dnnmg_mesh_t mesh, dnnmg_net_t net) {
    if (!mesh || !net) return -1;
    return 5 + (residual_cf_supported(mesh->g, mesh->info.precision) ? 1 : 0) +
           (mesh->info.P ? gru_launch_count(*net) : 0);
}

}  // extern "C"

namespace dnnmg {
cudaError_t launch_gru(const Net &net, const void *X, void *h, void *d, int P, cudaStream_t st) {
    if (net.tc) return launch_gru_tc(net, X, h, d, P, st);
    return launch_gru_cuda_core(net, X, h, d, P, st);
}
int gru_launch_count(const Net &) { return 1; }
}  // namespace dnnmg

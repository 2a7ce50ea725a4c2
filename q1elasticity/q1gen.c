/*
 * Q1 hexahedral linear-elasticity generator: the seeded synthetic inputs of
 * both the CUDA path and the oracle.  It holds none of the multigrid method's
 * arithmetic; it only builds the linear system A u = f (the paper's Eq. 1),
 * the six rigid-body modes B (the n x 6 near-nullspace matrix of Sec. 2) and
 * the material field.
 *
 * Mesh: nx x ny x nz cube elements of side h, node (i,j,k) at (i h, j h, k h),
 * node index i + (nx+1)(j + (ny+1) k) (x fastest), DOFs node-major (ux,uy,uz).
 * Element: trilinear Q1, 2x2x2 Gauss quadrature (exact for a cube).
 * Material: isotropic, lambda = E nu/((1+nu)(1-2nu)), mu = E/(2(1+nu)),
 * one E per element.
 * Dirichlet (clamp at x = 0): the clamped DOFs stay in the system with an
 * identity diagonal block; every off-diagonal block in their rows and columns
 * is structurally absent and their right-hand side is zero.
 *
 * The matrix is emitted as BSR with dense 3x3 blocks (all nine scalars of a
 * present block are stored, zeros included), int32 row_ptr/col, columns
 * ascending within each block row, values row-major per block.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off (no FMA contraction, so the
 * same input bits come out on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += golden gamma, then
 * the variant-13 finaliser of MurmurHash3.  Used for the inclusion centres. */
static uint64_t sm64_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double sm64_uniform(uint64_t *s) /* [0,1) with 53 random bits */
{
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t q1_splitmix64(uint64_t state, uint64_t *next_state)
{
    uint64_t s = state;
    uint64_t z = sm64_next(&s);
    if (next_state) *next_state = s;
    return z;
}

static inline int64_t node_id(int i, int j, int k, int nx, int ny)
{
    return (int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)(ny + 1) * k);
}

/* Element stiffness of a cube of side h with E = 1, Poisson ratio nu.
 * Local node a = ax + 2 ay + 4 az, (ax,ay,az) in {0,1}^3.
 * K[(a,i),(b,j)] = int lambda d_i N_a d_j N_b + mu d_j N_a d_i N_b
 *                      + mu delta_ij grad N_a . grad N_b  dV            */
void q1_element_stiffness(double h, double nu, double *Ke /* 24 x 24 */)
{
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    const double g = 1.0 / sqrt(3.0);
    const double gp[2] = {-g, g};
    const double jac = 2.0 / h;               /* d(xi)/dx               */
    const double wdet = (h / 2.0) * (h / 2.0) * (h / 2.0); /* weight 1 x det J */
    memset(Ke, 0, sizeof(double) * 24 * 24);
    for (int qz = 0; qz < 2; ++qz)
        for (int qy = 0; qy < 2; ++qy)
            for (int qx = 0; qx < 2; ++qx) {
                double xi[3] = {gp[qx], gp[qy], gp[qz]};
                double dN[8][3];
                for (int a = 0; a < 8; ++a) {
                    double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0,
                                   (a & 4) ? 1.0 : -1.0};
                    double f[3];
                    for (int d = 0; d < 3; ++d) f[d] = 1.0 + s[d] * xi[d];
                    dN[a][0] = 0.125 * s[0] * f[1] * f[2] * jac;
                    dN[a][1] = 0.125 * f[0] * s[1] * f[2] * jac;
                    dN[a][2] = 0.125 * f[0] * f[1] * s[2] * jac;
                }
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) {
                        double gg = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] +
                                    dN[a][2] * dN[b][2];
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) {
                                double v = lam * dN[a][i] * dN[b][j] +
                                           mu * dN[a][j] * dN[b][i];
                                if (i == j) v += mu * gg;
                                Ke[(3 * a + i) * 24 + 3 * b + j] += v * wdet;
                            }
                    }
            }
    /* mirror the upper triangle so that the assembled matrix is bitwise symmetric */
    for (int p = 0; p < 24; ++p)
        for (int q = p + 1; q < 24; ++q) Ke[q * 24 + p] = Ke[p * 24 + q];
}

/* Per-element Young's modulus: E_mat everywhere, E_inc inside seeded spheres
 * of radius r whose centres are uniform in the box [0,nx h]x[0,ny h]x[0,nz h];
 * an element is inside if its centroid is.  Spheres are added until the
 * volume fraction of inclusion elements reaches frac.  Returns the number of
 * spheres placed (or -1 if 100000 spheres did not reach the fraction). */
int q1_inclusions(int nx, int ny, int nz, double h, double r, double frac,
                  double E_mat, double E_inc, uint64_t seed, double *E_el)
{
    int64_t ne = (int64_t)nx * ny * nz, n_in = 0;
    for (int64_t e = 0; e < ne; ++e) E_el[e] = E_mat;
    if (frac <= 0.0) return 0;
    uint64_t s = seed;
    const double Lx = nx * h, Ly = ny * h, Lz = nz * h;
    for (int sphere = 0; sphere < 100000; ++sphere) {
        double cx = sm64_uniform(&s) * Lx, cy = sm64_uniform(&s) * Ly,
               cz = sm64_uniform(&s) * Lz;
        int i0 = (int)floor((cx - r) / h) - 1, i1 = (int)ceil((cx + r) / h) + 1;
        int j0 = (int)floor((cy - r) / h) - 1, j1 = (int)ceil((cy + r) / h) + 1;
        int k0 = (int)floor((cz - r) / h) - 1, k1 = (int)ceil((cz + r) / h) + 1;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (k0 < 0) k0 = 0;
        if (i1 > nx) i1 = nx;
        if (j1 > ny) j1 = ny;
        if (k1 > nz) k1 = nz;
        for (int k = k0; k < k1; ++k)
            for (int j = j0; j < j1; ++j)
                for (int i = i0; i < i1; ++i) {
                    double x = (i + 0.5) * h - cx, y = (j + 0.5) * h - cy,
                           z = (k + 0.5) * h - cz;
                    int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                    if (x * x + y * y + z * z <= r * r && E_el[e] != E_inc) {
                        E_el[e] = E_inc;
                        ++n_in;
                    }
                }
        if ((double)n_in >= frac * (double)ne) return sphere + 1;
    }
    return -1;
}

/* Block-row lengths of the 27-point node pattern (with the clamp rule).
 * row_ptr has (nx+1)(ny+1)(nz+1)+1 entries.  Returns nnzb. */
int64_t q1_pattern(int nx, int ny, int nz, int clamp, int32_t *row_ptr)
{
    int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1), cnt = 0;
    row_ptr[0] = 0;
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int64_t I = node_id(i, j, k, nx, ny);
                int c = 0;
                if (clamp && i == 0) {
                    c = 1;
                } else {
                    for (int dk = -1; dk <= 1; ++dk)
                        for (int dj = -1; dj <= 1; ++dj)
                            for (int di = -1; di <= 1; ++di) {
                                int a = i + di, b = j + dj, d = k + dk;
                                if (a < 0 || b < 0 || d < 0 || a > nx || b > ny || d > nz)
                                    continue;
                                if (clamp && a == 0) continue;
                                ++c;
                            }
                }
                cnt += c;
                if (cnt > 2147483647LL) return -1;
                row_ptr[I + 1] = (int32_t)cnt;
            }
    (void)nn;
    return cnt;
}

static int find_col(const int32_t *col, int32_t lo, int32_t hi, int32_t J)
{
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (col[mid] < J) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Fill col[] and val[] (nnzb x 9) given row_ptr from q1_pattern. */
int q1_assemble(int nx, int ny, int nz, double h, double nu, const double *E_el,
                int clamp, const int32_t *row_ptr, int32_t *col, double *val)
{
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int64_t I = node_id(i, j, k, nx, ny);
                int32_t p = row_ptr[I];
                if (clamp && i == 0) {
                    col[p] = (int32_t)I;
                    continue;
                }
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            int a = i + di, b = j + dj, d = k + dk;
                            if (a < 0 || b < 0 || d < 0 || a > nx || b > ny || d > nz)
                                continue;
                            if (clamp && a == 0) continue;
                            col[p++] = (int32_t)node_id(a, b, d, nx, ny);
                        }
                if (p != row_ptr[I + 1]) return -1;
            }
    int64_t nnzb = row_ptr[(int64_t)(nx + 1) * (ny + 1) * (nz + 1)];
    memset(val, 0, sizeof(double) * 9 * (size_t)nnzb);
    double Ke[24 * 24];
    q1_element_stiffness(h, nu, Ke);
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex) {
                double E = E_el[ex + (int64_t)nx * (ey + (int64_t)ny * ez)];
                int64_t g[8];
                int clamped[8];
                for (int a = 0; a < 8; ++a) {
                    int ix = ex + (a & 1), iy = ey + ((a >> 1) & 1), iz = ez + ((a >> 2) & 1);
                    g[a] = node_id(ix, iy, iz, nx, ny);
                    clamped[a] = clamp && ix == 0;
                }
                for (int a = 0; a < 8; ++a) {
                    if (clamped[a]) continue;
                    for (int b = 0; b < 8; ++b) {
                        if (clamped[b]) continue;
                        int32_t pos = find_col(col, row_ptr[g[a]], row_ptr[g[a] + 1],
                                               (int32_t)g[b]);
                        double *blk = val + 9 * (int64_t)pos;
                        for (int r = 0; r < 3; ++r)
                            for (int c = 0; c < 3; ++c)
                                blk[3 * r + c] += E * Ke[(3 * a + r) * 24 + 3 * b + c];
                    }
                }
            }
    if (clamp) {
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j) {
                int64_t I = node_id(0, j, k, nx, ny);
                double *blk = val + 9 * (int64_t)row_ptr[I];
                blk[0] = blk[4] = blk[8] = 1.0;
            }
    }
    return 0;
}

/* Node coordinates (nn x 3) and the six rigid-body modes B (3 nn x 6, row
 * major): columns tx, ty, tz, then rotations about x, y, z of the
 * coordinates relative to the mesh centroid:
 * rx = (0,-z,y), ry = (z,0,-x), rz = (-y,x,0). */
void q1_rigid_body_modes(int nx, int ny, int nz, double h, double *coords, double *B)
{
    const double cx = 0.5 * nx * h, cy = 0.5 * ny * h, cz = 0.5 * nz * h;
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int64_t I = node_id(i, j, k, nx, ny);
                double x = i * h, y = j * h, z = k * h;
                if (coords) {
                    coords[3 * I] = x;
                    coords[3 * I + 1] = y;
                    coords[3 * I + 2] = z;
                }
                double X = x - cx, Y = y - cy, Z = z - cz;
                double *b0 = B + 18 * I;
                double rows[3][6] = {{1, 0, 0, 0, Z, -Y},
                                     {0, 1, 0, -Z, 0, X},
                                     {0, 0, 1, Y, -X, 0}};
                memcpy(b0, rows, sizeof rows);
            }
}

/* Consistent load vector.  Body force (bx,by,bz) per unit volume: each of an
 * element's 8 nodes receives b h^3 / 8 (the integral of N_a b).  Traction
 * (tx,ty,tz) per unit area on the face x = nx h: each node of a boundary quad
 * receives t h^2 / 4.  Clamped DOFs get zero. */
void q1_load(int nx, int ny, int nz, double h, const double *body, const double *trac,
             int clamp, double *f)
{
    int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    memset(f, 0, sizeof(double) * 3 * (size_t)nn);
    if (body) {
        double w = h * h * h / 8.0;
        for (int ez = 0; ez < nz; ++ez)
            for (int ey = 0; ey < ny; ++ey)
                for (int ex = 0; ex < nx; ++ex)
                    for (int a = 0; a < 8; ++a) {
                        int64_t I = node_id(ex + (a & 1), ey + ((a >> 1) & 1),
                                            ez + ((a >> 2) & 1), nx, ny);
                        for (int d = 0; d < 3; ++d) f[3 * I + d] += body[d] * w;
                    }
    }
    if (trac) {
        double w = h * h / 4.0;
        for (int ez = 0; ez < nz; ++ez)
            for (int ey = 0; ey < ny; ++ey)
                for (int a = 0; a < 4; ++a) {
                    int64_t I = node_id(nx, ey + (a & 1), ez + ((a >> 1) & 1), nx, ny);
                    for (int d = 0; d < 3; ++d) f[3 * I + d] += trac[d] * w;
                }
    }
    if (clamp) {
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j) {
                int64_t I = node_id(0, j, k, nx, ny);
                f[3 * I] = f[3 * I + 1] = f[3 * I + 2] = 0.0;
            }
    }
}

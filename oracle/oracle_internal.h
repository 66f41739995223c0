// Internal declarations shared by the oracle's own translation units (test infrastructure).
#ifndef SGS_ORACLE_INTERNAL_H
#define SGS_ORACLE_INTERNAL_H
#include <cstdint>
#include <functional>
#include <vector>

#include "oracle.h"

namespace orc32 {
struct Support {
    bool visible;
    uint32_t depth_bits;
    float px, py, qa, qb, qc;
    float radius;  // ceil(3 sqrt(lambda_max)), pixels
};
Support support_of(const orc_scene* s, int64_t i, const float* cam);
bool in_support(const Support& g, int x, int y);
}  // namespace orc32

namespace orc64 {

struct Cam64 {
    double V[12];
    double campos[3];
    double fx, fy, cx, cy;
    int W, H;
};
Cam64 cam64(const float* c);

// Everything the forward computes for one (view, Gaussian) record, kept for the adjoint.
struct Pre64 {
    bool visible;          // FP32 cull (mirror)
    uint32_t depth_bits;   // FP32 view depth bits (mirror), the blend order key
    orc32::Support sup;    // FP32 support test data (mirror)
    double X[3], t[3];
    double qraw[4], qnorm, q[4];
    double R[3][3], s[3], M[3][3], Sig[3][3];
    double limx, limy, u, v;  // clamped x/z, y/z
    bool clampx, clampy;
    double J00, J02, J11, J12;
    double Tm[2][3];
    double a, b, c, det, A, B, C;
    double px, py;
    double dvec[3], dlen, dir[3];
    double pre[3], rgb[3];
    double opacity;
    int sh_top;  // highest SH band the record sums (adaptive degree, else sh_degree)
};
Pre64 preprocess(const orc_scene* s, int64_t i, const float* cam);

// Lobe frame of the orthogonal-frame mode from its 3 parameters f: the unit quaternion
// q = (1, f) / |(1, f)| and its rotation matrix R (lobe k's axis is column k).  Returns
// |(1, f)|.
double lobe_frame(const double f[3], double q[4], double R[3][3]);
// Lobe k's unit axis for any axis mode (0 free, 1 world, 2 frame) of Gaussian i.
void lobe_axis(const orc_scene* s, int64_t i, int lobe, double mu[3]);

// Real SH basis (Condon-Shortley phase), and its gradient w.r.t. the ambient direction.
double sh_basis(int l, int m, const double d[3]);
void sh_basis_grad(int l, int m, const double d[3], double g[3]);

// Per pixel: the ordered list of records whose support holds the pixel centre.
struct Hit {
    uint32_t depth_bits;
    int64_t i;
};
std::vector<Hit> support_list(const std::vector<Pre64>& pre, int x, int y);
double power64(const Pre64& p, int x, int y);

void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& fn);
}  // namespace orc64
#endif

// pd_damage: broken-bond counts and damage index (Eq. 12, 44, 48-49, 65).
//
// The paper writes d = 1 - lam (lam * omega0) / beta0 as a convolution with the
// characteristic influence function omega0 (Eq. 48-49, 65). The counts are
// integers, so they are evaluated here as the same convolution summed
// directly over the horizon offsets in integer arithmetic: exact, and cheaper
// than an FFT round trip for |H| <= a few hundred. beta is the node's number
// of in-body bonds (Eq. 12 restricted to B by the EC cut of Eq. 75).
#include "pd_plan.cuh"

namespace pd {

template <typename T>
__global__ void k_damage(int n1, int n2, int n3, const int *off, int cnt, const uint8_t *chi,
                         const uint8_t *lam, int32_t *nb, T *d, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    int beta = 0, k = 0;
    if (chi[p]) {
        const int lp = lam[p] != 0;
        for (int c = 0; c < cnt; ++c) {
            const int a = (i1 + off[3 * c]) & (n1 - 1);
            const int b = (i2 + off[3 * c + 1]) & (n2 - 1);
            const int e = (i3 + off[3 * c + 2]) & (n3 - 1);
            const int64_t q = ((int64_t)e * n2 + b) * n1 + a;
            if (!chi[q]) continue;
            ++beta;
            k += !(lp && lam[q]);
        }
    }
    if (nb) nb[p] = k;
    if (d) d[p] = beta ? (T)k / (T)beta : T(0);
}

}  // namespace pd

using namespace pd;

extern "C" pd_status pd_damage(pd_plan *p, const uint8_t *lambda, int32_t *nb, void *d, void *stream)
{
    if (!p || !lambda) {
        set_error("pd_damage: null plan or lambda");
        return PD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb_blk = (unsigned)((p->N + 255) / 256);
    if (p->prob.fp64)
        k_damage<double><<<nb_blk, 256, 0, st>>>(p->n1, p->n2, p->n3, p->hdev.off, p->hdev.cnt, p->chi, lambda, nb,
                                                  (double *)d, p->N);
    else
        k_damage<float><<<nb_blk, 256, 0, st>>>(p->n1, p->n2, p->n3, p->hdev.off, p->hdev.cnt, p->chi, lambda, nb,
                                                 (float *)d, p->N);
    PD_LAUNCH_CHECK();
    p->launches++;
    return PD_OK;
}

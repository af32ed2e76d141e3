// Host-side check of the library's termination rule (the one its device-side
// refinement loop runs): reads cases from stdin, prints one decision per case.
// Each case: k litmax mode tr_wider Cr Ce Rmax rmax_r abs_rel_tol eps_w bnorm
// anorm xnorm, then rh[0..k], then dh[0..k-1].  Test infrastructure only.
#include <cstdio>
#include <vector>

#include "../paper_2311_14616_gb300/csrc/ir_internal.cuh"

int main() {
    int k;
    while (std::scanf("%d", &k) == 1) {
        ir::TermArgs t;
        double bnorm, anorm, xnorm;
        if (std::scanf("%d %d %d %lf %lf %lf %lf %lf %lf %lf %lf %lf", &t.litmax, &t.mode, &t.tr_wider, &t.Cr, &t.Ce,
                       &t.Rmax, &t.rmax_r, &t.abs_rel_tol, &t.eps_w, &bnorm, &anorm, &xnorm) != 12)
            return 1;
        std::vector<double> rh(k + 1), dh(k > 0 ? k : 1);
        for (int i = 0; i <= k; ++i)
            if (std::scanf("%lf", &rh[i]) != 1) return 1;
        for (int i = 0; i < k; ++i)
            if (std::scanf("%lf", &dh[i]) != 1) return 1;
        std::printf("%d\n", ir::term_rule(rh.data(), dh.data(), k, bnorm, t, anorm, xnorm));
    }
    return 0;
}

/* A force-gradient HMC chain through the C ABI alone (plain C99).
 *
 *   cc -std=c99 -I include paper_0910_2950_gb300/examples/hmc_chain.c \
 *      -L paper_0910_2950_gb300 -l:libfg_lattice.so \
 *      -Wl,-rpath,paper_0910_2950_gb300 -o hmc_chain
 *   ./hmc_chain [L] [trajectories]
 *
 * Pure-gauge SU(3) Wilson action on an L^4 lattice (default 8) at beta = 6.0,
 * FP32 links and forces: a Haar-random start drawn on the device, then
 * trajectories of length 1 with the force-gradient integrator of Table 1 at
 * dt = 1/8, each with fresh Gaussian momenta and a Metropolis test.  Prints
 * dH, the accept decision and the mean plaquette per trajectory; exits
 * non-zero on any library error or a non-finite dH.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "fg_lattice.h"

static int check(fg_lattice *h, fg_status s, const char *what) {
  if (s == FG_OK) return 0;
  fprintf(stderr, "%s failed (status %d): %s\n", what, (int)s, h ? fg_last_error(h) : "");
  return 1;
}

int main(int argc, char **argv) {
  const int L = argc > 1 ? atoi(argv[1]) : 8;
  const int ntraj = argc > 2 ? atoi(argv[2]) : 10;
  fg_params p;
  fg_lattice *h = NULL;
  int i, accepted = 0, rc = 0;

  if (check(NULL, fg_params_default(&p), "fg_params_default")) return 1;
  for (i = 0; i < 4; ++i) p.dims[i] = L;
  p.beta = 6.0;
  p.precision = FG_FP32;
  p.seed = 2009;
  if (check(NULL, fg_lattice_create(&p, &h), "fg_lattice_create")) return 1;
  if (check(h, fg_random_gauge(h), "fg_random_gauge")) rc = 1;

  for (i = 0; !rc && i < ntraj; ++i) {
    fg_traj_result r;
    double plaq = 0.0;
    /* the first trajectories thermalise the hot start: accept them all */
    const double u = i < ntraj / 2 ? 0.0 : -1.0;
    if (check(h, fg_trajectory(h, FG_FORCE_GRADIENT, 0.125, 1.0, 1, u, &r), "fg_trajectory") ||
        check(h, fg_plaquette(h, &plaq), "fg_plaquette")) {
      rc = 1;
      break;
    }
    if (!isfinite(r.dH)) {
      fprintf(stderr, "non-finite dH at trajectory %d\n", i);
      rc = 1;
      break;
    }
    accepted += r.accepted;
    printf("trajectory %3d  dH %+.6e  accepted %d  forces %d  plaquette %.6f\n", i, r.dH, r.accepted,
           r.n_force, plaq);
  }
  if (!rc) printf("accepted %d of %d\n", accepted, ntraj);
  fg_lattice_destroy(h);
  return rc;
}

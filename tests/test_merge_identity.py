"""The identity the FP64 merge relies on (no GPU needed).

An event's gradient is stats_to_grad(st_i, S1_i) / S1_i (plus constants), and the merge
sums it over the events as stats_to_grad(sum_i st_i / S1_i, n) with n the number of
events: exact when stats_to_grad is linear in (st, S1) jointly.  This compiles the
library's own stats_to_grad for the host (nvcc; the program makes no CUDA call) and checks
the identity on random statistics and coefficients for both mass models and every
mixture-bound case (lambda_sigma = -1, 0, +1; for the multi-peak model also lam1_sigma).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "gwc_internal.cuh"
#include <cmath>
#include <cstdio>
#include <random>
using namespace gwc;
int main() {
  std::mt19937_64 rng(20260523);
  std::uniform_real_distribution<double> U(-1.0, 1.0), P(0.1, 2.0);
  int bad = 0, checked = 0;
  double worst = 0.0;
  for (int mp = 0; mp < 2; ++mp)
    for (int sig = -1; sig <= 1; ++sig)
      for (int sig1 = (mp ? -1 : 0); sig1 <= (mp ? 1 : 0); ++sig1) {
        LamD D{};
        D.mp = mp;
        D.lam_sigma = sig;
        D.lam1_sigma = sig1;
        double* co[] = {&D.invH0, &D.dZPa, &D.dZPmin, &D.dZPmax, &D.dZGmin, &D.dZGmax, &D.dZGmu,
                        &D.dZGsig, &D.inv_sig, &D.inv_lam, &D.inv_1ml, &D.gpk_inv1zp, &D.dZG2min,
                        &D.dZG2max, &D.dZG2mu, &D.dZG2sig, &D.inv_sig2, &D.inv_lam1, &D.inv_1ml1};
        for (double* c : co) *c = U(rng) * 3.0;
        const int npk = n_params(mp != 0);
        const int n_ev = 9;
        double direct[NP_MAX] = {0.0}, norm[NP_MAX] = {0.0};
        for (int e = 0; e < n_ev; ++e) {
          const double S1 = 10.0 * P(rng);
          double st[NP_MAX], G[NP_MAX];
          for (int i = 0; i < npk; ++i) st[i] = U(rng) * S1;
          stats_to_grad(st, S1, D, G);
          for (int i = 0; i < npk; ++i) {
            direct[i] += G[i] / S1;
            norm[i] += st[i] / S1;
          }
        }
        double merged[NP_MAX];
        stats_to_grad(norm, (double)n_ev, D, merged);
        for (int i = 0; i < npk; ++i) {
          const double d = std::fabs(merged[i] - direct[i]) / (1.0 + std::fabs(direct[i]));
          worst = d > worst ? d : worst;
          ++checked;
          if (d > 1e-12) ++bad;
        }
      }
  std::printf("%d %d %.3e\n", checked, bad, worst);
  return bad != 0;
}
"""


def test_events_gradient_sums_by_linearity(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "identity.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "identity"
    csrc = os.path.join(ROOT, "paper_2605_23538_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", csrc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad, worst = out.stdout.split()
    print(f"stats_to_grad linearity: {checked} components, worst relative difference {worst}")
    # 3 bound cases x 13 components (single peak), 3 x 3 cases x 16 (multi-peak)
    assert out.returncode == 0 and int(bad) == 0 and int(checked) == 3 * 13 + 9 * 16

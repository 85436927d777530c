// Host-side check of the hand-written reverse passes hllc_vjp and weno5_vjp
// (paper_2203_13760_gb300/csrc/vjp_math.cuh) against central differences of
// the forward functions, on random states (subsonic and supersonic, so that
// every HLLC branch is met).  Built and run by tests/test_vjp_math_host.py.
#include <cstdio>
#include <cmath>
#include <random>
#include "vjp_math.cuh"
using namespace jf;
template <int D> double check_hllc(std::mt19937_64& rng, double speed) {
  std::uniform_real_distribution<double> U(0, 1);
  Gas<double> g{}; g.gamma = 1.4; g.gm1 = 0.4; g.inv_gm1 = 2.5; g.inv_R = 1; g.mu = 0; g.lambda = 0; g.eps = 1e-6; g.safe = 0;
  double WL[5] = {0.2 + 2*U(rng), speed*(2*U(rng)-1), speed*(2*U(rng)-1), speed*(2*U(rng)-1), 0.2+2*U(rng)};
  double WR[5] = {0.2 + 2*U(rng), speed*(2*U(rng)-1), speed*(2*U(rng)-1), speed*(2*U(rng)-1), 0.2+2*U(rng)};
  double Fb[5]; for (auto& x : Fb) x = 2*U(rng)-1;
  double WLb[5], WRb[5]; hllc_vjp<double, D>(WL, WR, g, Fb, WLb, WRb);
  double worst = 0;
  for (int side = 0; side < 2; ++side) for (int k = 0; k < 5; ++k) {
    double h = 1e-6; double A[5], B[5], Fp[5], Fm[5];
    for (int i=0;i<5;++i){A[i]=WL[i];B[i]=WR[i];}
    double* X = side ? B : A; double x0 = X[k];
    X[k] = x0 + h; hllc<double, D>(A, B, g, Fp);
    X[k] = x0 - h; hllc<double, D>(A, B, g, Fm);
    double fd = 0; for (int q=0;q<5;++q) fd += Fb[q]*(Fp[q]-Fm[q])/(2*h);
    double ad = side ? WRb[k] : WLb[k];
    worst = std::fmax(worst, std::fabs(fd-ad)/(1+std::fabs(fd)));
  }
  return worst;
}
int main() {
  std::mt19937_64 rng(1);
  double w = 0;
  for (int t = 0; t < 2000; ++t) { w = std::fmax(w, check_hllc<0>(rng, 0.5)); w = std::fmax(w, check_hllc<1>(rng, 3.0)); w = std::fmax(w, check_hllc<2>(rng, 1.5)); }
  printf("hllc worst rel err %.3e\n", w);
  std::uniform_real_distribution<double> U(0, 1);
  double ww = 0;
  for (int t = 0; t < 2000; ++t) {
    double v[5]; for (auto& x : v) x = (t % 3 == 0) ? 2*U(rng) : 1.0 + 0.01*U(rng);
    double yb = 2*U(rng)-1; double vb[5] = {0,0,0,0,0};
    weno5_vjp(v[0],v[1],v[2],v[3],v[4],1e-6,yb,vb);
    for (int k = 0; k < 5; ++k) {
      double h = 1e-7, a[5], b[5]; for(int i=0;i<5;++i){a[i]=v[i];b[i]=v[i];} a[k]+=h; b[k]-=h;
      double fd = yb*(weno5(a[0],a[1],a[2],a[3],a[4],1e-6) - weno5(b[0],b[1],b[2],b[3],b[4],1e-6))/(2*h);
      ww = std::fmax(ww, std::fabs(fd - vb[k])/(1+std::fabs(fd)));
    }
  }
  printf("weno worst rel err %.3e\n", ww);
}

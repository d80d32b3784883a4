// D2Q37 model constants for the CUDA path.
//
// Velocity set (Sec. 3, Fig. "streamscheme": 37 populations hopping up to three sites):
// the integer vectors of the eight shells (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1)
// under sign changes and x<->y swap.  Population order: 0 = rest; 1..18 = the
// representatives below (vx > 0, or vx == 0 and vy > 0); 18 + k = -(vector k).
//
// Weights and lattice scale c: the paper defers them to its references; they are the
// unique positive solution of the lattice isotropy conditions
//   sum_i w_i (c vx_i)^p (c vy_i)^q = <Z^p><Z^q>,  (p,q) in {(0,0),(2,0),(4,0),(2,2),
//   (6,0),(4,2),(8,0),(6,2),(4,4)},  Z standard normal (reference temperature 1),
// solved to 40 digits and rounded here; lbm_model() exports them so the tests can
// check the conditions independently.
#pragma once

namespace d2q37 {

constexpr int Q = 37;
constexpr int NPAIR = 18;
constexpr double D = 2.0;

constexpr double C = 1.196979770393074358972388463853275434844;
constexpr double C2 = C * C;

// representative k = 1..18: (vx, vy)
__host__ __device__ constexpr int rep_vx(int k) {
  constexpr int t[19] = {0, 1, 0, 1, 1, 2, 0, 2, 1, 2, 1, 2, 2, 3, 0, 3, 1, 3, 1};
  return t[k];
}
__host__ __device__ constexpr int rep_vy(int k) {
  constexpr int t[19] = {0, 0, 1, 1, -1, 0, 2, 1, 2, -1, -2, 2, -2, 0, 3, 1, 3, -1, -3};
  return t[k];
}
__host__ __device__ constexpr int vx(int i) { return i == 0 ? 0 : (i <= 18 ? rep_vx(i) : -rep_vx(i - 18)); }
__host__ __device__ constexpr int vy(int i) { return i == 0 ? 0 : (i <= 18 ? rep_vy(i) : -rep_vy(i - 18)); }
__host__ __device__ constexpr int v2(int i) { return vx(i) * vx(i) + vy(i) * vy(i); }

// shell index 0..7 of |v|^2 in {0, 1, 2, 4, 5, 8, 9, 10}
__host__ __device__ constexpr int shell_of_v2(int q) {
  return q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 4 ? 3 : q == 5 ? 4 : q == 8 ? 5 : q == 9 ? 6 : 7;
}
__host__ __device__ constexpr int shell(int i) { return shell_of_v2(v2(i)); }
__host__ __device__ constexpr int shell_v2(int s) {
  constexpr int t[8] = {0, 1, 2, 4, 5, 8, 9, 10};
  return t[s];
}

__host__ __device__ constexpr double w_shell(int s) {
  constexpr double t[8] = {
      0.2331506691323525022865067040668499509961,     // (0,0)
      0.107306091542219002412464287183139935851,      // (1,0)
      0.05766785988879488203006921539333941471077,    // (1,1)
      0.01420821615845075026469894234413445497343,    // (2,0)
      0.005353049000513775232731501662188493535094,   // (2,1)
      0.001011937592673575475410908506639114714702,   // (2,2)
      0.0002453010277577173454659166432678444638839,  // (3,0)
      0.0002834142529941982174005252941948802334792,  // (3,1)
  };
  return t[s];
}
__host__ __device__ constexpr double weight(int i) { return w_shell(shell(i)); }

// |xi|^2 = c^2 |v|^2 of shell s
__host__ __device__ constexpr double q_shell(int s) { return C2 * (double)shell_v2(s); }

}  // namespace d2q37

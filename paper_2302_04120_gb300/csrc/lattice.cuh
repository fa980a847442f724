// Velocity sets shared by the CUDA kernels (device side only).
#pragma once

namespace lbmk {

// D2Q9 velocity set, Eqs. velocity_D2Q9 / weights_D2Q9
__host__ __device__ constexpr int cx9(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : (q == 3 || q == 6 || q == 7) ? -1 : 0; }
__host__ __device__ constexpr int cy9(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : (q == 4 || q == 7 || q == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp9(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 3) % 4) + 5); }
template <typename R> __host__ __device__ constexpr R w9(int q) { return q == 0 ? R(4) / R(9) : (q <= 4 ? R(1) / R(9) : R(1) / R(36)); }
// D2Q5 velocity set (extension: thermal LBE on five velocities)
__host__ __device__ constexpr int cx5(int q) { return q == 1 ? 1 : (q == 3 ? -1 : 0); }
__host__ __device__ constexpr int cy5(int q) { return q == 2 ? 1 : (q == 4 ? -1 : 0); }
__host__ __device__ constexpr int opp5(int q) { return q == 0 ? 0 : ((q + 1) % 4) + 1; }
template <typename R> __host__ __device__ constexpr R w5(int q) { return q == 0 ? R(1) / R(3) : R(1) / R(6); }

// mirror of a direction across a side normal to x (mx) or to y (my)
__host__ __device__ constexpr int mx9(int q) { return q == 1 ? 3 : q == 3 ? 1 : q == 5 ? 6 : q == 6 ? 5 : q == 7 ? 8 : q == 8 ? 7 : q; }
__host__ __device__ constexpr int my9(int q) { return q == 2 ? 4 : q == 4 ? 2 : q == 5 ? 8 : q == 8 ? 5 : q == 6 ? 7 : q == 7 ? 6 : q; }
__host__ __device__ constexpr int mx5(int q) { return q == 1 ? 3 : q == 3 ? 1 : q; }
__host__ __device__ constexpr int my5(int q) { return q == 2 ? 4 : q == 4 ? 2 : q; }

// The thermal lattice: QT = 5 (D2Q5) or 9 (the paper's D2Q9)
__host__ __device__ constexpr int cxT(int QT, int q) { return QT == 9 ? cx9(q) : cx5(q); }
__host__ __device__ constexpr int cyT(int QT, int q) { return QT == 9 ? cy9(q) : cy5(q); }
__host__ __device__ constexpr int oppT(int QT, int q) { return QT == 9 ? opp9(q) : opp5(q); }
template <typename R> __host__ __device__ constexpr R wT(int QT, int q) { return QT == 9 ? w9<R>(q) : w5<R>(q); }

static_assert(my9(7) == 6 && my9(8) == 5 && mx9(5) == 6 && mx9(8) == 7, "mirrors");
static_assert(opp9(1) == 3 && opp9(2) == 4 && opp9(3) == 1 && opp9(4) == 2, "opp9 axes");
static_assert(opp9(5) == 7 && opp9(6) == 8 && opp9(7) == 5 && opp9(8) == 6, "opp9 diagonals");
static_assert(opp5(1) == 3 && opp5(2) == 4 && opp5(3) == 1 && opp5(4) == 2, "opp5");

template <int PREC> struct Prec;
template <> struct Prec<0> { typedef double S; typedef double R; };
template <> struct Prec<1> { typedef float S; typedef float R; };

}  // namespace lbmk

// Generated by gen_tables.py -- do not edit.
// Degree-Q Gauss-Hermite velocity sets; constants rounded once to double.
#pragma once

namespace lbm {

struct D2Q37 {
  static constexpr int Q = 37;
  static constexpr int D = 2;
  static constexpr int NEQ = 4;
  static constexpr int NSHELL = 8;
  static constexpr double c = 0x1.326d4427cfd50p+0;   // 1.1969797703930743589723885
  static constexpr double c2 = 0x1.6ec9659248e55p+0;  // c^2 rounded once
  // e[i] = (e_x, e_y, e_z); i = 0 rest, then (e, -e) pairs
  static constexpr int e[37][3] = {
    {0, 0, 0},
    {1, 0, 0},
    {-1, 0, 0},
    {0, 1, 0},
    {0, -1, 0},
    {1, 1, 0},
    {-1, -1, 0},
    {1, -1, 0},
    {-1, 1, 0},
    {2, 0, 0},
    {-2, 0, 0},
    {0, 2, 0},
    {0, -2, 0},
    {2, 1, 0},
    {-2, -1, 0},
    {2, -1, 0},
    {-2, 1, 0},
    {1, 2, 0},
    {-1, -2, 0},
    {1, -2, 0},
    {-1, 2, 0},
    {2, 2, 0},
    {-2, -2, 0},
    {2, -2, 0},
    {-2, 2, 0},
    {3, 0, 0},
    {-3, 0, 0},
    {0, 3, 0},
    {0, -3, 0},
    {3, 1, 0},
    {-3, -1, 0},
    {3, -1, 0},
    {-3, 1, 0},
    {1, 3, 0},
    {-1, -3, 0},
    {1, -3, 0},
    {-1, 3, 0},
  };
  static constexpr int shell[37] = {0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7, 7};
  // |e|^2 of each shell
  static constexpr int shell_e2[8] = {0, 1, 2, 4, 5, 8, 9, 10};
  static constexpr double shell_w[8] = {
    0x1.dd7e1917b6364p-3,  // 0.2331506691323525022865067
    0x1.b786979d5dd9dp-4,  // 0.1073060915422190024124643
    0x1.d86a448815fd3p-5,  // 0.0576678598887948820300692
    0x1.d19327de15f21p-7,  // 0.0142082161584507502646989
    0x1.5ed142641e9d8p-8,  // 0.0053530490005137752327315
    0x1.0945fb76e9ba5p-10,  // 0.0010119375926735754754109
    0x1.01377e4533417p-12,  // 0.0002453010277577173454659
    0x1.292e6f2a5028ap-12,  // 0.0002834142529941982174005
  };
  static constexpr double w[37] = {
    0x1.dd7e1917b6364p-3,
    0x1.b786979d5dd9dp-4,
    0x1.b786979d5dd9dp-4,
    0x1.b786979d5dd9dp-4,
    0x1.b786979d5dd9dp-4,
    0x1.d86a448815fd3p-5,
    0x1.d86a448815fd3p-5,
    0x1.d86a448815fd3p-5,
    0x1.d86a448815fd3p-5,
    0x1.d19327de15f21p-7,
    0x1.d19327de15f21p-7,
    0x1.d19327de15f21p-7,
    0x1.d19327de15f21p-7,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.5ed142641e9d8p-8,
    0x1.0945fb76e9ba5p-10,
    0x1.0945fb76e9ba5p-10,
    0x1.0945fb76e9ba5p-10,
    0x1.0945fb76e9ba5p-10,
    0x1.01377e4533417p-12,
    0x1.01377e4533417p-12,
    0x1.01377e4533417p-12,
    0x1.01377e4533417p-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
    0x1.292e6f2a5028ap-12,
  };
  // element accessors usable in device code inside constant expressions
  __host__ __device__ static constexpr int E(int i, int a) { return e[i][a]; }
  __host__ __device__ static constexpr int SH(int i) { return shell[i]; }
  __host__ __device__ static constexpr int E2(int s) { return shell_e2[s]; }
  __host__ __device__ static constexpr double W(int i) { return w[i]; }
};

struct D3Q39 {
  static constexpr int Q = 39;
  static constexpr int D = 3;
  static constexpr int NEQ = 3;
  static constexpr int NSHELL = 6;
  static constexpr double c = 0x1.3988e1409212ep+0;   // 1.2247448713915890490986420
  static constexpr double c2 = 0x1.8000000000000p+0;  // c^2 rounded once
  // e[i] = (e_x, e_y, e_z); i = 0 rest, then (e, -e) pairs
  static constexpr int e[39][3] = {
    {0, 0, 0},
    {1, 0, 0},
    {-1, 0, 0},
    {0, 1, 0},
    {0, -1, 0},
    {0, 0, 1},
    {0, 0, -1},
    {1, 1, 1},
    {-1, -1, -1},
    {1, 1, -1},
    {-1, -1, 1},
    {1, -1, 1},
    {-1, 1, -1},
    {1, -1, -1},
    {-1, 1, 1},
    {2, 0, 0},
    {-2, 0, 0},
    {0, 2, 0},
    {0, -2, 0},
    {0, 0, 2},
    {0, 0, -2},
    {2, 2, 0},
    {-2, -2, 0},
    {2, 0, 2},
    {-2, 0, -2},
    {2, 0, -2},
    {-2, 0, 2},
    {2, -2, 0},
    {-2, 2, 0},
    {0, 2, 2},
    {0, -2, -2},
    {0, 2, -2},
    {0, -2, 2},
    {3, 0, 0},
    {-3, 0, 0},
    {0, 3, 0},
    {0, -3, 0},
    {0, 0, 3},
    {0, 0, -3},
  };
  static constexpr int shell[39] = {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5};
  // |e|^2 of each shell
  static constexpr int shell_e2[6] = {0, 1, 3, 4, 8, 9};
  static constexpr double shell_w[6] = {
    0x1.5555555555555p-4,  // 0.0833333333333333333333333
    0x1.5555555555555p-4,  // 0.0833333333333333333333333
    0x1.2f684bda12f68p-5,  // 0.0370370370370370370370370
    0x1.e573ac901e574p-7,  // 0.0148148148148148148148148
    0x1.2f684bda12f68p-9,  // 0.0023148148148148148148148
    0x1.43a2730abee4dp-11,  // 0.0006172839506172839506173
  };
  static constexpr double w[39] = {
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.5555555555555p-4,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.2f684bda12f68p-5,
    0x1.e573ac901e574p-7,
    0x1.e573ac901e574p-7,
    0x1.e573ac901e574p-7,
    0x1.e573ac901e574p-7,
    0x1.e573ac901e574p-7,
    0x1.e573ac901e574p-7,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.2f684bda12f68p-9,
    0x1.43a2730abee4dp-11,
    0x1.43a2730abee4dp-11,
    0x1.43a2730abee4dp-11,
    0x1.43a2730abee4dp-11,
    0x1.43a2730abee4dp-11,
    0x1.43a2730abee4dp-11,
  };
  // element accessors usable in device code inside constant expressions
  __host__ __device__ static constexpr int E(int i, int a) { return e[i][a]; }
  __host__ __device__ static constexpr int SH(int i) { return shell[i]; }
  __host__ __device__ static constexpr int E2(int s) { return shell_e2[s]; }
  __host__ __device__ static constexpr double W(int i) { return w[i]; }
};

}  // namespace lbm

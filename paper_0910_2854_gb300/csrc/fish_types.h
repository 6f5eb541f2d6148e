// fish_types.h -- host/device shared plain types of the sweep kernels.
#pragma once

namespace fish {

// sticky device status bits (reading C-16: no floor, report instead)
enum : unsigned { FLAG_RHO = 1u, FLAG_P = 2u, FLAG_NAN = 4u, FLAG_TIMEOUT = 8u };
enum : int { LIM_VANLEER = 0, LIM_MINMOD = 1, LIM_NONE = 2, LIM_HYBRID = 3 };
enum : int { BC_PERIODIC = 0, BC_OUTFLOW = 1 };

// Box geometry: cell counts n[axis], element strides st[axis] of the
// current memory layout, the axes in memory order from fastest to slowest
// (ord), and the boundary condition (0 periodic, 1 zeroth-order
// extrapolation).  Two layouts are used: x fastest (ord = x,y,z) for the y
// and z sweeps, and y fastest (ord = y,x,z) for the x sweeps.
struct Geom {
    int n[3];
    long long st[3];
    int ord[3];
    int bc;
};

}  // namespace fish

/*
 * hamr_oracle.h -- declarations shared by the two files of the FP64 CPU oracle
 * (hamr_oracle.c: the atomistic sLLG Heun step; hamr_ms_oracle.c: the multiscale window).
 * TEST INFRASTRUCTURE ONLY; nothing in the CUDA library includes this header.
 */
#pragma once
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KB 1.380649e-23 /* Boltzmann constant [J/K], exact SI value */
#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
    double ax, ay, az;         /* site spacing along x, y, z [m] */
    int32_t n_shells;          /* <= 4 */
    double shell_dist[4];      /* bond length of each shell [m] */
    double J[4];               /* exchange energy of each shell [J] */
    double mu_s;               /* atomic moment [J/T] */
    double ku;                 /* uniaxial anisotropy energy per atom [J], axis z */
    double alpha;              /* damping (the paper's lambda) */
    double dt;                 /* time step [s] */
    double gamma;              /* gyromagnetic ratio [rad/(s T)] */
    double T_amb, T_peak, fwhm, x0, y0, vx, vy; /* laser spot; fwhm <= 0: uniform T_amb */
    double B0, dir[3];         /* write-field amplitude [T] and direction */
    int32_t n_bits;            /* 0: static field B0*dir */
    const uint8_t *bits;       /* bit b = 1 -> polarity -1, 0 -> +1 */
    double bit_len, ramp_len, head_x0, head_v; /* [m], [m], [m], [m/s] */
    uint64_t seed;             /* Philox key of this replica */
} orc_params;


void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_thermal_normals(uint64_t seed, uint64_t site, uint64_t step, double xi[3]);
double orc_temperature(const orc_params *p, double x, double y, double t);
double orc_field_polarity(const orc_params *p, double t);
void orc_applied_field(const orc_params *p, double t, double B[3]);
void orc_llg_rhs(const orc_params *p, const double S[3], const double B[3], double f[3]);

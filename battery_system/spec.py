"""Constants of the synthetic layered thermal-battery system (one place for every reading).

The paper (Sec. 1.1) describes the coupled electrochemical physics but gives no
numbers for most coefficients; its matrices are snapshots of an unavailable
application.  Every value below is therefore a stated reading, chosen so that
the five-field system has the structure the paper describes: a solid potential
with Dirichlet on one collector and a unit current flux on the other
(Eq. solid-phase-voltage), a liquid potential with a small inductive mass term
and no boundary condition (Eq. liquid-phase-voltage), a linearised
Butler-Volmer point coupling between them (Eq. butler-volmer, beta = 0.5), a
Darcy pressure with storage (Eq. liquid-phase-continuity / liquid-velocity) and
two advected/diffused species (Eq. stefan-maxwell).
"""

# Butler-Volmer linearisation: k = a * i0 * alpha * F / (R * T)   (Eq. butler-volmer, beta = alpha = 0.5)
ALPHA = 0.5
FARADAY = 96485.0
GAS_R = 8.314
TEMPERATURE = 723.0          # molten-salt operating temperature (reading; the paper is silent)
SPECIFIC_AREA = 1.0          # a (reading)
DUDC = -0.05                 # U'(c1): open-circuit potential slope
I0_RANGE = (0.5, 2.0)        # exchange current, uniform per electrode cell; 0 in the separator

DT = 1.0e-3                  # time step
TAU_OVER_DT = 1.0e-3         # tau_I / dt: the small inductive term of the liquid potential
STORAGE_OVER_DT = 1.0        # s_p / dt: pressure storage (makes the p block nonsingular)
C0 = (1.0, 0.5)              # base concentrations c0_m of the two species (Newton term of A_{c,p})
GAMMA_P = 0.1                # stoichiometric factor of the reaction in the pressure row
GAMMA_C = (1.0, 0.0)         # stoichiometric factors in the species rows
EPS_CROSS = 1.0              # cross-species point coupling

# Layer means (anode, separator, cathode) of the lognormal fields, sigma_log = 0.5
SIGMA_S_MEANS = (1.0e2, 1.0e-2, 1.0e1)
KAPPA_E_MEAN = 1.0
PERM_MEAN = 1.0
PERM_Z_RATIO = 10.0          # K_z / K_x in 3D
DIFF_MEANS = (1.0, 0.5)      # D_1, D_2
LOG_SIGMA = 0.5

# Field ids and the block Gauss-Seidel order of the workload: [phi_s, phi_e] -> p -> [c1, c2]
PHI_S, PHI_E, PRESS, C1, C2 = 0, 1, 2, 3, 4
FIELD_NAMES = ("phi_s", "phi_e", "p", "c1", "c2")
NFIELDS = 5
WORKLOAD_ORDER = (PHI_S, PHI_E, PRESS, C1, C2)
# The paper's own order: non-voltage first (p, then species), then phi_e, then phi_s (Eqs. 2.6-2.8)
PAPER_ORDER = (PRESS, C1, C2, PHI_E, PHI_S)

# RNG streams of the counter-based generator
STREAM_SIGMA, STREAM_KAPPA, STREAM_PERM, STREAM_D1, STREAM_D2, STREAM_I0, STREAM_RHS = 1, 2, 3, 4, 5, 6, 7

# Named workloads: (dim, nx, ny, nz, layer axis, repeats along z)
CONFIGS = {
    "C1": dict(dim=2, nx=64, ny=64, nz=1, stack=False),
    "C2": dict(dim=3, nx=64, ny=64, nz=64, stack=False),
    "C3": dict(dim=3, nx=48, ny=48, nz=48, stack=False),
    "C4": dict(dim=3, nx=128, ny=128, nz=128, stack=False),
    "C5": dict(dim=3, nx=160, ny=160, nz=400, stack=True),
}
STACK_PERIOD = 20            # cells per anode/separator/cathode repeat along z (C5), 20 repeats


def bv_rate_constant():
    """k / i0 = a * alpha * F / (R T)."""
    return SPECIFIC_AREA * ALPHA * FARADAY / (GAS_R * TEMPERATURE)

"""Physical constants and synthetic chemistry for the workloads.

Species molar masses and standard molar enthalpies of formation are the usual tabulated values
(298 K, ideal gas). The reaction constants below are SYNTHETIC and chosen for this benchmark:
the paper's two-step mechanisms (Section 3.1 for propane, Section 3.2.2 for methane) cite their
constants to other work that is not available here. They give a methane-like lean flame whose
thickness spans a few cells at the workloads' grid spacings; they are not a validated mechanism.
"""

# atomic masses (kg/mol); molar masses are built from them so that every reaction balances mass
_ATOM = {"C": 12.011e-3, "H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}
_COMPOSITION = {"CH4": {"C": 1, "H": 4}, "O2": {"O": 2}, "CO": {"C": 1, "O": 1}, "CO2": {"C": 1, "O": 2},
                "H2O": {"H": 2, "O": 1}, "N2": {"N": 2}}


def _molar_mass(name):
    return sum(_ATOM[a] * n for a, n in _COMPOSITION[name].items())


# name: (molar mass kg/mol, molar enthalpy of formation J/mol)
_THERMO = {n: (_molar_mass(n), h) for n, h in
           (("CH4", -74.87e3), ("O2", 0.0), ("CO", -110.53e3), ("CO2", -393.52e3), ("H2O", -241.83e3), ("N2", 0.0))}
# lumped product of CH4 + 2 O2 -> CO2 + 2 H2O, counted as 3 moles of "P"
_THERMO["P"] = ((_THERMO["CO2"][0] + 2 * _THERMO["H2O"][0]) / 3.0, (-393.52e3 - 2 * 241.83e3) / 3.0)

# constant Lewis numbers (synthetic round values)
_LEWIS = {"CH4": 1.0, "O2": 1.1, "CO": 1.1, "CO2": 1.4, "H2O": 0.8, "N2": 1.0, "P": 1.0}


# Heat capacities c_p,k(T) = a0 + a1 T (J/(kg K)) for the variable-thermodynamics option: SYNTHETIC
# round values that follow the rise of each species' c_p between 300 and 1500 K, in the NASA
# polynomial's place (the paper's thermochemistry library and its data are not available). The
# lumped product P mixes CO2 and H2O by mass (44 : 36).
_CP_LINEAR = {"CH4": (1590.0, 2.14), "O2": (863.0, 0.19), "CO": (985.0, 0.183), "CO2": (730.0, 0.4),
              "H2O": (1685.0, 0.6), "N2": (990.0, 0.167), "P": (1160.0, 0.49)}


def variable_cp(cfg):
    """Switch a configuration to temperature-dependent species heat capacities (in place)."""
    cfg["variable_cp"] = True
    cfg["T0_thermo"] = 298.15
    for s in cfg["species"]:
        a0, a1 = _CP_LINEAR[s["name"]]
        s["cp_poly"] = [a0, a1, 0.0, 0.0, 0.0]
    return cfg


def mixture_averaged(cfg):
    """Switch a configuration to mixture-averaged species diffusion (in place) with synthetic pair
    Lewis numbers Le_kj = sqrt(m_kj / m_N2N2), m_kj = W_k W_j / (W_k + W_j) the reduced molar mass
    (binary diffusivities of kinetic theory scale as m_kj^-1/2 at fixed collision diameter), so that
    the N2-N2 pair has Le = 1; e.g. CH4-N2 0.85, H2O-N2 0.89, O2-N2 1.03, CO2-N2 1.11."""
    Ws = [s["W"] for s in cfg["species"]]
    W_n2 = _molar_mass("N2")
    m_ref = W_n2 * W_n2 / (2.0 * W_n2)
    cfg["mixture_averaged"] = True
    cfg["Le_pair"] = [[(Wk * Wj / (Wk + Wj) / m_ref) ** 0.5 for Wj in Ws] for Wk in Ws]
    return cfg


def species(names, unity_lewis=False):
    out = []
    for n in names:
        W, hmol = _THERMO[n]
        out.append({"name": n, "W": W, "Le": 1.0 if unity_lewis else _LEWIS[n], "hf": hmol / W})
    return out


SPECIES = {"6sp": ["CH4", "O2", "CO", "CO2", "H2O", "N2"], "4sp": ["CH4", "O2", "P", "N2"]}


def chemistry_2step(A1=1.0e9, A2=5.0e6):
    """CH4 + 1.5 O2 -> CO + 2 H2O ; CO + 0.5 O2 -> CO2 (both irreversible), 6 species order."""
    return [
        {"A": A1, "beta": 0.0, "E": 1.4e5, "nu": {0: -1.0, 1: -1.5, 2: 1.0, 4: 2.0},
         "order": {0: 0.5, 1: 0.65}},
        {"A": A2, "beta": 0.0, "E": 5.0e4, "nu": {2: -1.0, 1: -0.5, 3: 1.0},
         "order": {2: 1.0, 1: 0.5}},
    ]


def chemistry_1step(A=1.0e9):
    """CH4 + 2 O2 -> 3 P (lumped products), 4 species order (CH4, O2, P, N2)."""
    return [{"A": A, "beta": 0.0, "E": 1.4e5, "nu": {0: -1.0, 1: -2.0, 2: 3.0},
             "order": {0: 0.5, 1: 0.65}}]


def mixture_phi(names, phi):
    """Unburnt CH4/air mass fractions at equivalence ratio phi (air = O2 + 3.76 N2)."""
    moles = {"CH4": phi, "O2": 2.0, "N2": 7.52}
    mass = {k: v * _THERMO[k][0] for k, v in moles.items()}
    tot = sum(mass.values())
    return [mass.get(n, 0.0) / tot for n in names]


def burnt_mixture(names, phi):
    """Complete-combustion products of the lean mixture (CO2, H2O or lumped P), mass fractions.

    Used only to build initial fields (hot pockets); the oracle pins compute the adiabatic
    state separately.
    """
    moles = {"O2": 2.0 - 2.0 * phi, "N2": 7.52}
    if "CO2" in names:
        moles.update({"CO2": phi, "H2O": 2.0 * phi})
    else:
        moles.update({"P": 3.0 * phi})
    mass = {k: v * _THERMO[k][0] for k, v in moles.items()}
    tot = sum(mass.values())
    return [mass.get(n, 0.0) / tot for n in names]

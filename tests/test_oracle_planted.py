"""The pins catch plausible mistakes: the oracle is rebuilt with one planted
mistake at a time (on the CPU) and at least one pin must fail.  Each check
below is one of the pins of test_oracle_pins.py, test_oracle_extensions.py,
test_oracle_symmetry.py or test_oracle_two_step.py, run against the mutant."""
import pytest

from paper_1611_08536_gb300 import inputs as I
from tests import test_oracle_extensions as ext
from tests import test_oracle_pins as pins
from tests import test_oracle_symmetry as sym
from tests import test_oracle_two_step as two

PLANTS = ["PLANT_DROP_UNSCATTERED", "PLANT_ABSORB_ONCE", "PLANT_SEGMENT_SIGN",
          "PLANT_HG_UNNORMALISED", "PLANT_MIRROR_INDEX", "PLANT_FRESNEL_SWAP",
          "PLANT_WRONG_DIRECTION_INDEX", "PLANT_POINT_OFF_BY_ONE", "PLANT_SENSOR_LAG_SIGN",
          "PLANT_SOURCE_FULL_PATH", "PLANT_HIGH_FACE_NO_FLIP",
          "PLANT_SNELL_INVERTED", "PLANT_TWO_STEP_PATH_MEDIUM1", "PLANT_TWO_STEP_NO_FLIP",
          "PLANT_HG_SIGN", "PLANT_HG_EXPONENT"]

CHECKS = [
    pins.test_axis_direction_single_target,
    pins.test_edge_direction_closed_form,
    pins.test_unscattered_survival_factor,
    pins.test_perpendicular_scatter_four_points,
    pins.test_isotropic_kernel_uniform,
    pins.test_hg_mean_cosine_slope_is_one,
    pins.test_hg_forward_limit,
    lambda o: pins.test_interior_column_sums_equal_absorption_survival(o, 10.0, 0.01, 0.9),
    pins.test_mirror_columns_sum_to_survival_everywhere,
    pins.test_energy_conservation_mirror_with_interface,
    pins.test_ballistic_axis_translation_exact,
    pins.test_fresnel_normal_incidence_at_edge,
    pins.test_total_internal_reflection_corner_direction,
    pins.test_interface_transmission_normal_incidence,
    pins.test_interface_split_oblique_edge_direction,
    ext.test_point_row_reads_the_state,
    ext.test_sensor_delayed_impulse_shifts,
    lambda o: ext.test_source_column_axis_closed_form(o, 0.25),
    lambda o: sym.test_homogeneous_cube_has_the_48_symmetries(o, I.MIRROR),
    two.test_mass_and_fresnel_share_oblique,
    two.test_snell_angle_of_the_transmitted_split,
    two.test_scattering_free_beam_lands_around_the_two_step_points,
    two.test_normal_incidence,
    two.test_absorption_along_the_two_path_pieces,
]


@pytest.mark.parametrize("plant", PLANTS)
def test_planted_mistake_is_caught(oracle_mod, plant):
    failed = []
    with oracle_mod.planted(plant):
        for chk in CHECKS:
            try:
                chk(oracle_mod)
            except (AssertionError, ValueError, RuntimeError):
                failed.append(getattr(chk, "__name__", "lambda"))
    assert failed, f"no pin caught {plant}"


def test_unplanted_oracle_passes_the_same_checks(oracle_mod):
    for chk in CHECKS:
        chk(oracle_mod)

"""The committed double-float tables equal a fresh run of their generator."""
import os
import subprocess
import sys

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1511_02166_gb300", "csrc")


def test_tables_regenerate_identically():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_df_tables.py")],
                         capture_output=True, text=True, check=True).stdout
    with open(os.path.join(CSRC, "df_tables.cuh")) as f:
        assert f.read() == out

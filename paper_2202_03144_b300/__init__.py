"""B300-native ptychographic reconstruction (ePIE, DM, LSQML) behind a C ABI."""

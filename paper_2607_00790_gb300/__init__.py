"""GB300-native WSBM / HSS entry generator (see include/wsbm_hss.h)."""
